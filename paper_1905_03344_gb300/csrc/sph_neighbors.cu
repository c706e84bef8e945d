// sph_neighbors.cu -- neighbour discovery, second half: symmetric neighbour
// lists in CSR form (Table 1 "Neighbour Discovery", symmetric union reading
// R11): j is in N(i) iff j != i and r_ij^2 < 4 h_i^2 or r_ij^2 < 4 h_j^2,
// with the minimum image along periodic z.  n_i = #{j : r_ij^2 < 4 h_i^2}
// feeds the smoothing-length adaptation.
//
// Each particle is served by a group of TPP lanes.  The group walks the
// (2K+1)^3 cells around the particle's cell, skipping cells whose box is
// farther than 2 max(h_i, h_max(cell)), and tests candidates in FP32 on
// cell-relative coordinates.  A candidate is decided in FP32 only outside a
// guard band around the threshold; inside it the FP64 predicate is evaluated
// with the same operation order and rounding as its definition, so the lists
// are bit-exact.
//
// One pass builds the CSR: a CTA takes the next tile of consecutive sorted
// particles (tile ids handed out in launch order by an atomic counter),
// stages each particle's row in shared memory (ordered by stencil cell, then
// by sorted index, through a ballot inside the group), scans the row lengths
// of the tile, and obtains the tile's global offset by a decoupled look-back
// over the preceding tiles' published sums.  The rows are then written with
// coalesced stores.  Rows longer than their shared-memory slot are recorded
// and written in full by a fix-up pass that repeats their search.  The
// look-back only waits for tiles handed out earlier (already running), and
// every wait is bounded: past the limit the kernel reports SPH_ETIMEOUT
// through the status word instead of spinning on.
#include "sph_internal.cuh"

namespace sphg {

constexpr int kNbThreads = 128;
constexpr int kNbSmemWords = 8192;                // 32 KB of staged rows per CTA
constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagPrefix = 2ull << 62;
constexpr unsigned long long kValMask = (1ull << 62) - 1ull;
constexpr long long kSpinLimit = 1ll << 24;

// exact FP64 predicate, no contraction: bit 0 union, bit 1 own radius
__device__ __forceinline__ int exact_pair(double xi, double yi, double zi, double hi, double xj,
                                          double yj, double zj, double hj, double lz)
{
    const double dx = __dsub_rn(xi, xj);
    const double dy = __dsub_rn(yi, yj);
    double dz = __dsub_rn(zi, zj);
    const double hl = __dmul_rn(0.5, lz);
    if (dz > hl) dz = __dsub_rn(dz, lz);
    else if (dz < -hl) dz = __dadd_rn(dz, lz);
    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    const int own = r2 < __dmul_rn(__dmul_rn(4.0, hi), hi);
    const int oth = r2 < __dmul_rn(__dmul_rn(4.0, hj), hj);
    return (own | oth) | (own << 1);
}

// distance from a point at cell-relative coordinate o in [0, s) to the cell
// offset by d cells along one axis
__device__ __forceinline__ float cell_gap(int d, float o, float s)
{
    float g = d > 0 ? (float)d * s - o : (d < 0 ? o - (float)(d + 1) * s : 0.0f);
    return fmaxf(g, 0.0f);
}

// The search for particle i by a group of TPP lanes.  emit(pos, word) is
// called by each lane holding a neighbour, pos being its index in the row;
// returns the row length (uniform in the group) and adds to own.
template <int TPP, class Emit>
__device__ __forceinline__ uint32_t search_row(const NbArgs& a, int64_t i, int gl, unsigned gmask,
                                               unsigned ltmask, uint32_t& own, Emit emit)
{
    const PatchDev* P = a.pd + a.g.patch_of[i];
    const float s_f = P->s_f, sz_f = P->sz_f, lz_f = P->lz_f;
    const int ncx = P->ncx, ncy = P->ncy, ncz = P->ncz, K = P->K, zmode = P->zmode;
    const int64_t cbase = P->cell_base;
    const float4 ri = a.r4[i];
    const uint32_t cc = a.g.cellxyz[i];
    const int cx = cc & 255, cy = (cc >> 8) & 255, cz = cc >> 16;
    const float hf = (float)a.h[i];
    const float Ti = ri.w;                                  // 4 h_i^2
    const float tol = kTolBase + kTolCell * (s_f / hf);
    const float flo = 1.0f - tol, fhi = 1.0f + tol;
    const float slack = (1.0f / 4096.0f) * s_f;
    const float Rg = 2.0f * fmaxf(hf, P->hmax_f) * (1.0f + 1.0f / 512.0f) + slack;
    const float Rg2 = Rg * Rg;
    uint32_t cnt = 0;
    const int nz = zmode ? ncz : 2 * K + 1;
    for (int iz = 0; iz < nz; iz++) {
        int czj, zd;
        float zsh, gz;
        if (zmode == 0) {
            const int dcz = iz - K;
            czj = cz + dcz;
            if (czj < 0) czj += ncz;
            else if (czj >= ncz) czj -= ncz;
            zsh = (float)dcz * sz_f;
            gz = cell_gap(dcz, ri.z, sz_f);
            zd = dcz + 2;
        } else {
            czj = cz + iz;
            if (czj >= ncz) czj -= ncz;
            zsh = (float)iz * sz_f;
            gz = 0.0f;
            zd = iz;
        }
        const float gz2 = gz * gz;
        if (gz2 >= Rg2) continue;
        const float zo = ri.z - zsh;
        for (int dcy = -K; dcy <= K; dcy++) {
            const int cyj = cy + dcy;
            if (cyj < 0 || cyj >= ncy) continue;
            const float gy = cell_gap(dcy, ri.y, s_f);
            const float gzy2 = fmaf(gy, gy, gz2);
            if (gzy2 >= Rg2) continue;
            const float yo = ri.y - (float)dcy * s_f;
            for (int dcx = -K; dcx <= K; dcx++) {
                const int cxj = cx + dcx;
                if (cxj < 0 || cxj >= ncx) continue;
                const float gx = cell_gap(dcx, ri.x, s_f);
                const float d2 = fmaf(gx, gx, gzy2);
                const int64_t lin = cbase + ((int64_t)czj * ncy + cyj) * ncx + cxj;
                const uint2 se = a.g.cse[lin];
                if (se.x >= se.y) continue;
                const float R = 2.0f * fmaxf(hf, a.g.chmax[lin]) * (1.0f + 1.0f / 512.0f) + slack;
                if (d2 >= R * R) continue;
                const float xo = ri.x - (float)dcx * s_f;
                const uint32_t kk = (uint32_t)((dcx + 2) + 5 * (dcy + 2) + 25 * zd) << kColBits;
                for (uint32_t jb = se.x; jb < se.y; jb += TPP) {
                    const uint32_t j = jb + gl;
                    bool in = false;
                    if (j < se.y) {
                        const float4 q = a.r4[j];
                        const float dx = xo - q.x, dy = yo - q.y;
                        float dz = zo - q.z;
                        if (zmode) {
                            if (dz > 0.5f * lz_f) dz -= lz_f;
                            else if (dz < -0.5f * lz_f) dz += lz_f;
                        }
                        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                        const float T = fmaxf(Ti, q.w);
                        if (r2 <= T * fhi && (int64_t)j != i) {
                            in = r2 < T * flo;
                            bool io = r2 < Ti * flo;
                            if (!in || (!io && r2 <= Ti * fhi)) {
                                const int e = exact_pair(a.x[i], a.y[i], a.z[i], a.h[i], a.x[j], a.y[j],
                                                         a.z[j], a.h[j], P->lz);
                                in = e & 1;
                                io = (e >> 1) & 1;
                            }
                            own += io;
                        }
                    }
                    const unsigned b = __ballot_sync(gmask, in);
                    if (in) emit(cnt + (uint32_t)__popc(b & ltmask), j | kk);
                    cnt += (uint32_t)__popc(b);
                }
            }
        }
    }
    return cnt;
}

template <int TPP>
__device__ __forceinline__ uint32_t group_sum_u32(uint32_t v, unsigned gmask)
{
#pragma unroll
    for (int o = TPP / 2; o > 0; o >>= 1) v += __shfl_xor_sync(gmask, v, o);
    return v;
}

__device__ __forceinline__ uint32_t block_excl_scan_u32(uint32_t v, uint32_t* total, uint32_t* sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t inc = v;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) sh[warp] = inc;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int w = 0; w < nw; w++) {
            const uint32_t c = sh[w];
            sh[w] = run;
            run += c;
        }
        sh[32] = run;
    }
    __syncthreads();
    const uint32_t r = inc - v + sh[warp];
    *total = sh[32];
    __syncthreads();
    return r;
}

template <int TPP>
__global__ void __launch_bounds__(kNbThreads) k_nb_single(NbArgs a)
{
    constexpr int PPT = kNbThreads / TPP;          // particles per tile
    constexpr int CAP = kNbSmemWords / PPT;        // staged row capacity
    __shared__ uint32_t s_list[kNbSmemWords];
    __shared__ uint32_t s_len[PPT];
    __shared__ uint32_t s_loc[PPT];
    __shared__ uint32_t s_scan[33];
    __shared__ uint32_t s_tile;
    __shared__ unsigned long long s_base;
    if (*a.status & kStBad) return;
    const int lane = threadIdx.x & 31;
    const int gl = lane & (TPP - 1);
    const unsigned gmask = TPP == 32 ? 0xffffffffu : (((1u << TPP) - 1u) << (lane & ~(TPP - 1)));
    const unsigned ltmask = (1u << lane) - 1u;
    const int slot = threadIdx.x / TPP;
    const int64_t ntiles = (a.n + PPT - 1) / PPT;
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(a.tile_counter, 1u);
        __syncthreads();
        const int64_t tile = s_tile;
        if (tile >= ntiles) break;
        const int64_t i = tile * PPT + slot;
        uint32_t own = 0, len = 0;
        if (i < a.n) {
            uint32_t* row = s_list + slot * CAP;
            len = search_row<TPP>(a, i, gl, gmask, ltmask, own, [&](uint32_t pos, uint32_t w) {
                if (pos < (uint32_t)CAP) row[pos] = w;
            });
        }
        own = group_sum_u32<TPP>(own, gmask);
        if (gl == 0) {
            s_len[slot] = len;
            if (i < a.n) {
                a.cnt[i] = len;
                a.nown[i] = own;
                if (len > (uint32_t)CAP) a.fix_list[atomicAdd(a.fix_count, 1u)] = (uint32_t)i;
            }
        }
        __syncthreads();
        uint32_t tot;
        const uint32_t ex = block_excl_scan_u32(threadIdx.x < PPT ? s_len[threadIdx.x] : 0u, &tot, s_scan);
        if (threadIdx.x < PPT) s_loc[threadIdx.x] = ex;
        if (threadIdx.x == 0) {
            // decoupled look-back: publish the tile sum, add predecessors' sums
            // until one with an inclusive prefix is found
            atomicExch(a.tile_state + tile, kFlagAgg | (unsigned long long)tot);
            unsigned long long excl = 0;
            long long spins = 0;
            bool ok = true;
            for (int64_t t = tile - 1; t >= 0;) {
                const unsigned long long w = *((volatile unsigned long long*)(a.tile_state + t));
                if ((w >> 62) == 0ull) {
                    if (++spins > kSpinLimit) {
                        ok = false;
                        break;
                    }
                    continue;
                }
                excl += w & kValMask;
                if ((w & kFlagPrefix) && !(w & kFlagAgg)) break;
                t--;
            }
            if (!ok) atomicOr(a.status, kStTimeout);
            atomicExch(a.tile_state + tile, kFlagPrefix | ((excl + tot) & kValMask));
            s_base = excl;
            if (tile == ntiles - 1) a.off_w[a.n] = excl + tot;
            if (excl + tot > (unsigned long long)a.max_pairs) atomicOr(a.status, kStOverflow);
        }
        __syncthreads();
        const unsigned long long base = s_base;
        const bool write = !(*((volatile int*)a.status) & (kStOverflow | kStTimeout));
        if (threadIdx.x < PPT && tile * PPT + threadIdx.x < a.n)
            a.off_w[tile * PPT + threadIdx.x] = base + s_loc[threadIdx.x];
        if (write) {
            // one warp per row, consecutive rows are adjacent in col[]
            const int warp = threadIdx.x >> 5, nw = kNbThreads >> 5;
            for (int p = warp; p < PPT; p += nw) {
                const uint32_t L = min(s_len[p], (uint32_t)CAP);
                const unsigned long long r0 = base + s_loc[p];
                for (uint32_t k = lane; k < L; k += 32) a.col[r0 + k] = s_list[p * CAP + k];
            }
        }
        __syncthreads();
    }
}

// rows that did not fit their shared-memory slot: search again, write whole row
template <int TPP>
__global__ void __launch_bounds__(256) k_nb_fixup(NbArgs a)
{
    if (*a.status & kStBad) return;
    const int lane = threadIdx.x & 31;
    const int gl = lane & (TPP - 1);
    const unsigned gmask = TPP == 32 ? 0xffffffffu : (((1u << TPP) - 1u) << (lane & ~(TPP - 1)));
    const unsigned ltmask = (1u << lane) - 1u;
    const uint32_t count = *a.fix_count;
    const int64_t gs = ((int64_t)gridDim.x * blockDim.x) / TPP;
    for (int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / TPP; q < count; q += gs) {
        const int64_t i = a.fix_list[q];
        const unsigned long long r0 = a.off_w[i];
        uint32_t own = 0;
        search_row<TPP>(a, i, gl, gmask, ltmask, own, [&](uint32_t pos, uint32_t w) {
            if (r0 + pos < (unsigned long long)a.max_pairs) a.col[r0 + pos] = w;
        });
    }
}

int launch_nb_lists(const Launch& L, const NbArgs& a, int tpp)
{
    if (a.n <= 0) {
        cudaMemsetAsync(a.off_w, 0, sizeof(uint64_t), L.stream);
        return 0;
    }
    const int grid = L.sms * 6;
    switch (tpp) {
    case 1: k_nb_single<1><<<grid, kNbThreads, 0, L.stream>>>(a); break;
    case 2: k_nb_single<2><<<grid, kNbThreads, 0, L.stream>>>(a); break;
    case 4: k_nb_single<4><<<grid, kNbThreads, 0, L.stream>>>(a); break;
    case 16: k_nb_single<16><<<grid, kNbThreads, 0, L.stream>>>(a); break;
    case 32: k_nb_single<32><<<grid, kNbThreads, 0, L.stream>>>(a); break;
    default: k_nb_single<8><<<grid, kNbThreads, 0, L.stream>>>(a); break;
    }
    return 1;
}

int launch_nb_fixup(const Launch& L, const NbArgs& a, int tpp)
{
    if (a.n <= 0) return 0;
    const int grid = L.sms * 2;
    switch (tpp) {
    case 1: k_nb_fixup<1><<<grid, 256, 0, L.stream>>>(a); break;
    case 2: k_nb_fixup<2><<<grid, 256, 0, L.stream>>>(a); break;
    case 4: k_nb_fixup<4><<<grid, 256, 0, L.stream>>>(a); break;
    case 16: k_nb_fixup<16><<<grid, 256, 0, L.stream>>>(a); break;
    case 32: k_nb_fixup<32><<<grid, 256, 0, L.stream>>>(a); break;
    default: k_nb_fixup<8><<<grid, 256, 0, L.stream>>>(a); break;
    }
    return 1;
}

int64_t nb_tile_words(int64_t n) { return n / 4 + 16; }

__global__ void k_unpack_cols(int64_t nnz, const uint32_t* col, uint32_t* out)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz;
         k += (int64_t)gridDim.x * blockDim.x)
        out[k] = col[k] & kColMask;
}

int launch_unpack_cols(const Launch& L, int64_t nnz, const uint32_t* col, uint32_t* out)
{
    if (nnz <= 0) return 0;
    int64_t blocks = (nnz + 255) / 256;
    if (blocks > (int64_t)L.sms * 16) blocks = (int64_t)L.sms * 16;
    k_unpack_cols<<<(unsigned)blocks, 256, 0, L.stream>>>(nnz, col, out);
    return 1;
}

}  // namespace sphg
