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
// are bit-exact.  Two passes (count, fill) around an exclusive scan keep the
// rows in a plain CSR layout; the fill pass orders each row by stencil cell,
// then by sorted index, via a ballot inside the group.
#include "sph_internal.cuh"

namespace sphg {

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

template <int TPP, bool FILL>
__global__ void __launch_bounds__(256) k_neighbors(NbArgs a)
{
    const int lane = threadIdx.x & 31;
    const int gl = lane & (TPP - 1);
    const unsigned gmask = TPP == 32 ? 0xffffffffu : (((1u << TPP) - 1u) << (lane & ~(TPP - 1)));
    const unsigned ltmask = (1u << lane) - 1u;
    const int64_t gs = ((int64_t)gridDim.x * blockDim.x) / TPP;
    if (*a.status & (kStOverflow | kStNonFinite)) return;  // no usable grid or list
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / TPP; i < a.n; i += gs) {
        const PatchDev* P = a.pd + a.g.patch_of[i];
        const float s_f = P->s_f, sz_f = P->sz_f, lz_f = P->lz_f;
        const int ncx = P->ncx, ncy = P->ncy, ncz = P->ncz, K = P->K, zmode = P->zmode;
        const int64_t cbase = P->cell_base;
        const float4 ri = a.r4[i];
        const uint32_t cc = a.g.cellxyz[i];
        const int cx = cc & 255, cy = (cc >> 8) & 255, cz = cc >> 16;
        const float hf = ri.w;
        const float Ti = 4.0f * hf * hf;
        const float tol = kTolBase + kTolCell * (s_f / hf);
        const float flo = 1.0f - tol, fhi = 1.0f + tol;
        const float slack = (1.0f / 4096.0f) * s_f;
        const float Rg = 2.0f * fmaxf(hf, P->hmax_f) * (1.0f + 1.0f / 512.0f) + slack;
        const float Rg2 = Rg * Rg;
        uint32_t cnt = 0, own = 0;
        uint64_t wpos = FILL ? a.off[i] : 0;
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
                    const uint32_t kk = (uint32_t)((dcx + 2) + 5 * (dcy + 2) + 25 * zd);
                    for (uint32_t jb = se.x; jb < se.y; jb += TPP) {
                        const uint32_t j = jb + gl;
                        bool in = false, io = false;
                        if (j < se.y && (int64_t)j != i) {
                            const float4 q = a.r4[j];
                            const float dx = xo - q.x, dy = yo - q.y;
                            float dz = zo - q.z;
                            if (zmode) {
                                if (dz > 0.5f * lz_f) dz -= lz_f;
                                else if (dz < -0.5f * lz_f) dz += lz_f;
                            }
                            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                            const float T = fmaxf(Ti, 4.0f * q.w * q.w);
                            in = r2 < T * flo;
                            io = r2 < Ti * flo;
                            if ((!in && r2 <= T * fhi) || (!io && r2 <= Ti * fhi)) {
                                const int e = exact_pair(a.x[i], a.y[i], a.z[i], a.h[i], a.x[j], a.y[j],
                                                         a.z[j], a.h[j], P->lz);
                                in = e & 1;
                                io = (e >> 1) & 1;
                            }
                        }
                        cnt += in;
                        own += io;
                        if (FILL) {
                            const unsigned b = __ballot_sync(gmask, in);
                            if (in) {
                                const uint64_t pos = wpos + (uint64_t)__popc(b & ltmask);
                                if (pos < (uint64_t)a.max_pairs) a.col[pos] = j | (kk << kColBits);
                            }
                            wpos += (uint64_t)__popc(b);
                        }
                    }
                }
            }
        }
        if (!FILL) {
#pragma unroll
            for (int o = TPP / 2; o > 0; o >>= 1) {
                cnt += __shfl_xor_sync(gmask, cnt, o);
                own += __shfl_xor_sync(gmask, own, o);
            }
            if (gl == 0) {
                a.cnt[i] = cnt;
                a.nown[i] = own;
            }
        }
    }
}

template <bool FILL>
static int launch_nb(const Launch& L, const NbArgs& a, int tpp)
{
    if (a.n <= 0) return 0;
    const int threads = 256;
    int64_t blocks = (a.n * tpp + threads - 1) / threads;
    const int64_t cap = (int64_t)L.sms * 8;
    if (blocks > cap) blocks = cap;
    switch (tpp) {
    case 1: k_neighbors<1, FILL><<<(unsigned)blocks, threads, 0, L.stream>>>(a); break;
    case 2: k_neighbors<2, FILL><<<(unsigned)blocks, threads, 0, L.stream>>>(a); break;
    case 4: k_neighbors<4, FILL><<<(unsigned)blocks, threads, 0, L.stream>>>(a); break;
    case 16: k_neighbors<16, FILL><<<(unsigned)blocks, threads, 0, L.stream>>>(a); break;
    case 32: k_neighbors<32, FILL><<<(unsigned)blocks, threads, 0, L.stream>>>(a); break;
    default: k_neighbors<8, FILL><<<(unsigned)blocks, threads, 0, L.stream>>>(a); break;
    }
    return 1;
}

int launch_nb_count(const Launch& L, const NbArgs& a, int tpp) { return launch_nb<false>(L, a, tpp); }
int launch_nb_fill(const Launch& L, const NbArgs& a, int tpp) { return launch_nb<true>(L, a, tpp); }

__global__ void k_check_capacity(const uint64_t* total, int64_t max_pairs, int* status)
{
    if (*total > (uint64_t)max_pairs) atomicOr(status, kStOverflow);
}

int launch_check_capacity(const Launch& L, const uint64_t* total, int64_t max_pairs, int* status)
{
    k_check_capacity<<<1, 1, 0, L.stream>>>(total, max_pairs, status);
    return 1;
}

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
