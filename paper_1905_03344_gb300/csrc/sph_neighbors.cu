// sph_neighbors.cu -- neighbour discovery, second half: the symmetric
// neighbour lists, one row per particle from the search in sph_walk.cuh.
//
// Rows go straight to the pool.  Each lane reserves its row before the walk,
// from the row-length hint c (the particle's row length in the previous
// lists) as c + c/3 + 8 entries -- on a lattice a small change of h adds a
// whole shell of neighbours at once, up to about a third of the row -- or,
// without a hint, from a first walk that only counts.  Reservations are
// rounded up to a multiple of 8 entries, so every row starts on a 32-byte
// boundary.  Hits collect in a 16-slot ring in shared memory and leave it as
// whole 32-byte sectors.  A row that outgrows its reservation is walked again
// into a fresh reservation of its exact (rounded) length.  Shared memory per
// warp is 2 KB, which leaves the SM's L1 to the candidate gathers.  Row
// contents are fixed by the inputs; only the place of a row in the pool
// depends on scheduling, and every consumer reads a row through its start
// and length, so all results are bitwise reproducible.  The canonical CSR
// with prefix offsets is built from the pool on demand (sph_get_neighbors).
#include "sph_pairmath.cuh"
#include "sph_walk.cuh"

namespace sphg {

// counting walk (col = nullptr) and repair walk (straight to the pool): one
// out-of-line copy serves both
template <int K, bool EXACT>
__device__ __noinline__ RowSink<kWalkFlat, EXACT> walk_all_flat(const NbArgs& a, const PatchDev* P, int64_t i,
                                                             bool big, RowSink<kWalkFlat, EXACT> row)
{
    walk_all<RowSink<kWalkFlat, EXACT>, K>(a, P, i, big, row);
    return row;
}

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v, int lane)
{
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// K: stencil half-extent, the same for every patch (it follows cell_factor);
// EXACT = false: the candidate superset (every candidate within the scaled
// search radius in FP32, no n_i)
template <int K, bool EXACT>
__global__ void __launch_bounds__(32 * kNbtWarps, SPH_NB_MINB) k_nb_thread(NbArgs a)
{
    extern __shared__ __align__(16) uint32_t nb_ring[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* ring = nb_ring + warp * (32 * (kRing + kPend)) + lane;
    if (*a.status & kStBad) return;
    const unsigned long long pool_cap = (unsigned long long)a.pool_cap;
    for (int64_t q = (int64_t)blockIdx.x * kNbtWarps + warp; q < a.nunits; q += (int64_t)gridDim.x * kNbtWarps) {
        const WorkItem U = a.units[q];
        const PatchDev* P = a.pd + U.patch;
        const int64_t i = U.begin + lane;
        const bool act = i < U.end;
        // big particles sit at the end of their patch
        const bool big = act && i >= P->end - (int64_t)P->nbig;
        // reservation: the hint plus a margin, or the counted length
        uint32_t res = 0;
        if (act) {
            const uint32_t hint = a.rowcap[i];
            if (hint == kNoHint) {
                const RowSink<kWalkFlat, EXACT> rc =
                    walk_all_flat<K, EXACT>(a, P, i, big, RowSink<kWalkFlat, EXACT>{nullptr, nullptr, 0u, 0u, 0u, 0u});
                res = round8(rc.cnt);
            } else {
                const uint32_t c = min(hint, (uint32_t)a.n);
                res = round8(c + c / 3u + kHintMargin);
            }
        }
        const uint32_t inc = warp_incl_scan(res, lane);
        const uint32_t tot = __shfl_sync(0xffffffffu, inc, 31);
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&a.pool_used[0], (unsigned long long)tot);
        base = __shfl_sync(0xffffffffu, base, 0);
        const bool ok = base + tot <= pool_cap;
        if (!ok && lane == 0) atomicOr(a.status, kStOverflow);
        unsigned long long r0 = base + (inc - res);
        RowSink<kWalkRing, EXACT> row = {a.col + r0, ring, ok ? res : 0u, 0u, 0u, 0u};
        if (act) {
            walk_all<RowSink<kWalkRing, EXACT>, K>(a, P, i, big, row);
            row.finish();
            // only a row that is in the pool (within the sink's reservation,
            // which is 0 for a warp whose reservation did not fit)
            if (row.npend > 0 && row.npend <= (uint32_t)kPend && row.cnt <= row.res) row.resolve_band(a, P, i);
        }
        if (act && ok && (row.cnt > res || row.npend > (uint32_t)kPend)) {
            // outgrew the reservation, or deferred more guard-band words than
            // it notes: walk again, deciding in place, into an exact reservation
            const uint32_t need = round8(row.cnt);
            r0 = atomicAdd(&a.pool_used[0], (unsigned long long)need);
            if (r0 + need <= pool_cap) {
                const RowSink<kWalkFlat, EXACT> rr = walk_all_flat<K, EXACT>(
                    a, P, i, big, RowSink<kWalkFlat, EXACT>{a.col + r0, nullptr, need, 0u, 0u, 0u});
                row.cnt = rr.cnt;
                row.own = rr.own;
            } else {
                atomicOr(a.status, kStOverflow);
            }
        }
        if (act) {
            a.rowstart[i] = r0;
            a.cnt[i] = row.cnt;
            if (EXACT) a.nown[i] = row.own;
        }
        const uint32_t listed = __shfl_sync(0xffffffffu, warp_incl_scan(act ? row.cnt : 0u, lane), 31);
        if (lane == 0) {
            const unsigned long long before = atomicAdd(&a.pool_used[1], (unsigned long long)listed);
            if (before + listed > (unsigned long long)a.max_pairs) atomicOr(a.status, kStOverflow);
        }
    }
}

template <int K, bool EXACT>
void launch_nb_thread(const Launch& L, const NbArgs& a)
{
    const size_t smem = sizeof(uint32_t) * 32 * (kRing + kPend) * kNbtWarps;
    static int per_sm = 0;
    if (!per_sm) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_nb_thread<K, EXACT>, 32 * kNbtWarps, smem);
        if (per_sm < 1) per_sm = 1;
        // shared memory only for the rings of the resident CTAs: the rest is L1
        int smem_max = 0, dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        if (smem_max > 0) {
            const size_t need = (size_t)per_sm * (smem + 1024);
            int pct = (int)((need * 100 + (size_t)smem_max - 1) / (size_t)smem_max);
            pct = pct < 1 ? 1 : (pct > 100 ? 100 : pct);
            cudaFuncSetAttribute(k_nb_thread<K, EXACT>, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
        }
    }
    k_nb_thread<K, EXACT><<<L.sms * per_sm, 32 * kNbtWarps, smem, L.stream>>>(a);
}

int launch_nb_lists(const Launch& L, const NbArgs& a, int K, int exact)
{
    if (a.n <= 0 || a.nunits <= 0) return 0;
    if (exact) {
        if (K == 1) launch_nb_thread<1, true>(L, a);
        else if (K == 2) launch_nb_thread<2, true>(L, a);
        else launch_nb_thread<3, true>(L, a);
    } else {
        if (K == 1) launch_nb_thread<1, false>(L, a);
        else if (K == 2) launch_nb_thread<2, false>(L, a);
        else launch_nb_thread<3, false>(L, a);
    }
    return 1;
}

// ---- exact lists from a reused candidate superset -------------------------
// Row i of the superset (col_s from rowstart[i], cnt_s[i] words, built on an
// earlier state with the search radius scaled by 1 + skin) is decided again
// on the current state: the FP32 test on the records refreshed for the
// current positions and h, and the exact FP64 predicate inside the guard
// band, as in the search.  The accepted words keep their order and go to
// the exact pool at the same offset.  A group of TPP lanes per row: each
// lane decides one word per round; the group ballots and writes the accepted
// words contiguously.  Groups of a warp run their rounds together (a shorter
// row idles through the longer one's last rounds), so TPP = 32: one row per
// warp in lockstep.
template <int TPP>
__global__ void __launch_bounds__(256) k_nb_filter(NbArgs a, const uint32_t* col_s, const uint32_t* cnt_s)
{
    if (*a.status & kStBad) return;
    const int lane = threadIdx.x & 31;
    const int gl = lane & (TPP - 1);
    const unsigned gmask = TPP == 32 ? 0xffffffffu : (((1u << TPP) - 1u) << (lane & ~(TPP - 1)));
    const unsigned below = (1u << lane) - 1u;    // lanes before this one
    const int64_t gs = ((int64_t)gridDim.x * blockDim.x) / TPP;
    unsigned long long listed = 0;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / TPP; i < a.n; i += gs) {
        const PatchDev* P = a.pd + a.g.patch_of[i];
        const float s_f = P->s_f, sz_f = P->sz_f, lz_f = P->lz_f;
        const int zmode = P->zmode, Dcode = zmode ? max(2, P->ncz) : 2;
        const float4 ri = a.r4[i];
        const uint32_t ci = a.g.cellxyz[i];
        const float Ti = ri.w;
        const float sh = s_f / (float)a.h[i];
        const unsigned long long rs = a.rowstart[i];
        const uint32_t len = cnt_s[i];
        uint32_t out = 0, own = 0;
        for (uint32_t k0 = 0; k0 < len; k0 += TPP) {
            const uint32_t k = k0 + (uint32_t)gl;
            bool in = false, io = false;
            uint32_t w = 0;
            if (k < len) {
                w = col_s[rs + k];
                const uint32_t j = w & kColMask;
                const float4 q = a.r4[j];
                const uint32_t code = w >> kColBits;
                float dx, dy, dz;
                int D;
                if (code != kFarCode) {
                    const float4 e = stencil_offset(code);
                    if (zmode) rel_dx<1>(e, s_f, sz_f, lz_f, (float)P->ncz, ri.x, ri.y, ri.z, q, dx, dy, dz);
                    else rel_dx<0>(e, s_f, sz_f, lz_f, (float)P->ncz, ri.x, ri.y, ri.z, q, dx, dy, dz);
                    D = Dcode;
                } else {
                    const uint32_t cj = a.g.cellxyz[j];
                    rel_dx_far(ci, cj, s_f, sz_f, lz_f, ri.x, ri.y, ri.z, q, dx, dy, dz);
                    const int ax = abs((int)(cj & 255u) - (int)(ci & 255u));
                    const int ay = abs((int)((cj >> 8) & 255u) - (int)((ci >> 8) & 255u));
                    const int az = abs((int)(cj >> 16) - (int)(ci >> 16));
                    D = max(ax, max(ay, az));
                }
                const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                const float T = fmaxf(Ti, q.w);
                const float tol = guard_tol(sh, D);
                const float fhi = 1.0f + tol;
                if (r2 <= T * fhi) {
                    const int d = pair_decision(a, P, i, j, r2, Ti, T, 1.0f - tol, fhi);
                    in = d & 1;
                    io = (d >> 1) & 1;
                }
            }
            const unsigned bin = __ballot_sync(gmask, in) & gmask;
            const unsigned bio = __ballot_sync(gmask, io) & gmask;
            if (in) a.col[rs + out + (uint32_t)__popc(bin & below)] = w;
            out += (uint32_t)__popc(bin);
            own += (uint32_t)__popc(bio);
        }
        if (gl == 0) {
            a.cnt[i] = out;
            a.nown[i] = own;
            listed += out;
        }
    }
    for (int o = 16; o > 0; o >>= 1) listed += __shfl_xor_sync(0xffffffffu, listed, o);
    if (lane == 0 && listed) {
        const unsigned long long before = atomicAdd(&a.pool_used[1], listed);
        if (before + listed > (unsigned long long)a.max_pairs) atomicOr(a.status, kStOverflow);
    }
}

int launch_nb_filter(const Launch& L, const NbArgs& a, const uint32_t* col_s, const uint32_t* cnt_s)
{
    if (a.n <= 0) return 0;
    constexpr int TPP = 32;
    int64_t blocks = (a.n * TPP + 255) / 256;
    if (blocks > (int64_t)L.sms * 8) blocks = (int64_t)L.sms * 8;
    k_nb_filter<TPP><<<(unsigned)blocks, 256, 0, L.stream>>>(a, col_s, cnt_s);
    return 1;
}

// canonical CSR: row i of the pool, columns without the stencil bits, to
// out[off[i] ..]; one warp per row
__global__ void k_canonical_rows(int64_t n, const unsigned long long* rowstart, const uint32_t* cnt,
                                 const uint64_t* off, const uint32_t* col, uint32_t* out)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
        const unsigned long long r0 = rowstart[i];
        const uint64_t o = off[i];
        for (uint32_t k = lane; k < cnt[i]; k += 32) out[o + k] = col[r0 + k] & kColMask;
    }
}

int launch_canonical_rows(const Launch& L, int64_t n, const unsigned long long* rowstart,
                          const uint32_t* cnt, const uint64_t* off, const uint32_t* col, uint32_t* out)
{
    if (n <= 0) return 0;
    int64_t blocks = (n * 32 + 255) / 256;
    if (blocks > (int64_t)L.sms * 16) blocks = (int64_t)L.sms * 16;
    k_canonical_rows<<<(unsigned)blocks, 256, 0, L.stream>>>(n, rowstart, cnt, off, col, out);
    return 1;
}

}  // namespace sphg
