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
#include "sph_walk.cuh"

namespace sphg {

// counting walk (col = nullptr) and repair walk (straight to the pool): one
// out-of-line copy serves both
template <int K>
__device__ __noinline__ RowSink<kWalkFlat> walk_all_flat(const NbArgs& a, const PatchDev* P, int64_t i, bool big,
                                                      RowSink<kWalkFlat> row)
{
    walk_all<RowSink<kWalkFlat>, K>(a, P, i, big, row);
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

// K: stencil half-extent, the same for every patch (it follows cell_factor)
template <int K>
__global__ void __launch_bounds__(32 * kNbtWarps, SPH_NB_MINB) k_nb_thread(NbArgs a)
{
    extern __shared__ __align__(16) uint32_t nb_ring[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* ring = nb_ring + warp * (32 * kRing) + lane;
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
                const RowSink<kWalkFlat> rc = walk_all_flat<K>(a, P, i, big, RowSink<kWalkFlat>{nullptr, nullptr, 0u, 0u, 0u});
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
        RowSink<kWalkRing> row = {a.col + r0, ring, ok ? res : 0u, 0u, 0u};
        if (act) {
            walk_all<RowSink<kWalkRing>, K>(a, P, i, big, row);
            row.finish();
        }
        if (act && ok && row.cnt > res) {
            // outgrew the reservation: walk again into an exact one
            const uint32_t need = round8(row.cnt);
            r0 = atomicAdd(&a.pool_used[0], (unsigned long long)need);
            if (r0 + need <= pool_cap) {
                walk_all_flat<K>(a, P, i, big, RowSink<kWalkFlat>{a.col + r0, nullptr, need, 0u, 0u});
            } else {
                atomicOr(a.status, kStOverflow);
            }
        }
        if (act) {
            a.rowstart[i] = r0;
            a.cnt[i] = row.cnt;
            a.nown[i] = row.own;
        }
        const uint32_t listed = __shfl_sync(0xffffffffu, warp_incl_scan(act ? row.cnt : 0u, lane), 31);
        if (lane == 0) {
            const unsigned long long before = atomicAdd(&a.pool_used[1], (unsigned long long)listed);
            if (before + listed > (unsigned long long)a.max_pairs) atomicOr(a.status, kStOverflow);
        }
    }
}

template <int K>
void launch_nb_thread(const Launch& L, const NbArgs& a)
{
    const size_t smem = sizeof(uint32_t) * 32 * kRing * kNbtWarps;
    static int per_sm = 0;
    if (!per_sm) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_nb_thread<K>, 32 * kNbtWarps, smem);
        if (per_sm < 1) per_sm = 1;
        // shared memory only for the rings of the resident CTAs: the rest is L1
        int smem_max = 0, dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        if (smem_max > 0) {
            const size_t need = (size_t)per_sm * (smem + 1024);
            int pct = (int)((need * 100 + (size_t)smem_max - 1) / (size_t)smem_max);
            pct = pct < 1 ? 1 : (pct > 100 ? 100 : pct);
            cudaFuncSetAttribute(k_nb_thread<K>, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
        }
    }
    k_nb_thread<K><<<L.sms * per_sm, 32 * kNbtWarps, smem, L.stream>>>(a);
}

int launch_nb_lists(const Launch& L, const NbArgs& a, int K)
{
    if (a.n <= 0 || a.nunits <= 0) return 0;
    if (K == 1) launch_nb_thread<1>(L, a);
    else if (K == 2) launch_nb_thread<2>(L, a);
    else launch_nb_thread<3>(L, a);
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
