// sph_fused.cuh -- the list-free pair sums: the density (with the EOS) and
// the momentum and energy sums evaluated inside the neighbour search, with
// no neighbour lists in memory.
//
// Each kernel walks the candidates of every particle exactly as the list
// builder does (the walks of sph_walk.cuh, one thread per particle, a warp
// per 32 consecutive sorted particles of one patch) and hands the decided
// pairs to a sink that accumulates the sum instead of writing a row.  The
// pair set is therefore the lists' set (the union decision is the same FP32
// test with the same exact FP64 predicate inside the guard band), and the
// pairs arrive in row order; the per-pair arithmetic is the same functions
// the list sums call (sph_pairmath.cuh).  The density pass also counts
// |N(i)| and n_i, which the smoothing-length update reads, so a step needs
// no list at all.  With one lane per particle the sums over the lists and
// these sums give the same bits.
//
// The momentum sink queues the accepted column words in a per-lane ring in
// shared memory and evaluates them four at a time -- the chunk of four row
// words the list sum takes -- at the end of each candidate group, so the
// pair arithmetic appears once per walk rather than once per unrolled
// candidate.
//
// The cost is the search itself, paid in both passes: the lists are written
// once and read twice, the search is run twice.  sph_autotune times both.
#pragma once
#include "sph_pairmath.cuh"
#include "sph_walk.cuh"

namespace sphg {

#ifndef SPH_FUSED_DEN_MINB
#define SPH_FUSED_DEN_MINB 6            // resident 128-thread CTAs per SM (density pass)
#endif
#ifndef SPH_FUSED_MOM_MINB
#define SPH_FUSED_MOM_MINB 4            // resident 128-thread CTAs per SM (momentum pass)
#endif

constexpr int kQueue = 8;               // queue slots per lane
static_assert(kGroup + 3 <= kQueue, "a group's pairs and the three left over must fit the queue");

// the union decision alone (the momentum pass needs no n_i): a candidate
// the walk passed has r2 <= T (1 + tol); below T (1 - tol) it is in,
// inside the band the FP64 predicate decides
__device__ __forceinline__ bool union_decision(const NbArgs& a, const PatchDev* P, int64_t i, uint32_t j, float r2,
                                               float T, float flo)
{
    if (r2 < T * flo) return true;
    return (exact_pair_at(a, i, j, P->lz) & 1) != 0;
}

// ---- mixed precision --------------------------------------------------------
template <int KERN, bool GH>
struct DensSink {
    PairSrc src;
    PairSide I;
    float inv2h;
    int kn, zmode;
    float sum, comp, sumd, compd;
    uint32_t cnt, own;

    __device__ __forceinline__ uint32_t mark() const { return 0u; }
    __device__ __forceinline__ void group_end(uint32_t) {}
    __device__ __forceinline__ void decide(const NbArgs& a, const PatchDev* P, int64_t i, uint32_t j, float r2,
                                           float Ti, float T, float flo, float fhi, uint32_t w)
    {
        const int d = pair_decision(a, P, i, j, r2, Ti, T, flo, fhi);
        own += (uint32_t)(d >> 1);
        if (!(d & 1)) return;
        cnt++;
        const float4 q = src.r5[j];
        if (zmode) density_pair<1, KERN, GH>(src, I, inv2h, kn, w, q, q.w, sum, comp, sumd, compd);
        else density_pair<0, KERN, GH>(src, I, inv2h, kn, w, q, q.w, sum, comp, sumd, compd);
    }
};

template <int KERN, bool GH>
struct MomSink {
    PairSrc src;
    PairSide I;
    float4 vi, ti;
    float wi5;
    MomConst K;
    int kn, zmode;
    uint32_t* q;             // this lane's queue: slot k at q[32 k]
    uint32_t head, tail;     // words evaluated, words queued
    MomAcc A;

    __device__ __forceinline__ uint32_t mark() const { return 0u; }
    __device__ __forceinline__ void decide(const NbArgs& a, const PatchDev* P, int64_t i, uint32_t j, float r2,
                                           float, float T, float flo, float, uint32_t w)
    {
        if (!union_decision(a, P, i, j, r2, T, flo)) return;
        q[32 * (tail & (kQueue - 1))] = w;
        tail++;
    }
    // the next nv (<= 4) queued words as one chunk
    __device__ __forceinline__ void chunk(uint32_t nv)
    {
        const uint32_t cws[4] = {q[32 * (head & (kQueue - 1))], q[32 * ((head + 1) & (kQueue - 1))],
                                 q[32 * ((head + 2) & (kQueue - 1))], q[32 * ((head + 3) & (kQueue - 1))]};
        float bx, by, bz, bu;
        const GlobalRecs R{src};
        if (zmode) momentum_chunk<1, KERN, GH>(src, I, vi, ti, wi5, K, kn, cws, nv, bx, by, bz, bu, R);
        else momentum_chunk<0, KERN, GH>(src, I, vi, ti, wi5, K, kn, cws, nv, bx, by, bz, bu, R);
        mom_acc_add(A, bx, by, bz, bu);
        head += nv;
    }
    // a group adds at most kGroup words to at most three left over: one chunk
    // brings the queue back below four
    __device__ __forceinline__ void group_end(uint32_t)
    {
        if (tail - head >= 4u) chunk(4u);
    }
    __device__ __forceinline__ void finish()
    {
        if (tail != head) chunk(tail - head);
    }
};

// ---- FP64 -------------------------------------------------------------------
template <int KERN, bool GH>
struct DensSinkD {
    const PairArgs* pa;
    double xi, yi, zi, w, lz;
    int kn;
    double sum, sumd;
    uint32_t cnt, own;

    __device__ __forceinline__ uint32_t mark() const { return 0u; }
    __device__ __forceinline__ void group_end(uint32_t) {}
    __device__ __forceinline__ void decide(const NbArgs& a, const PatchDev* P, int64_t i, uint32_t j, float r2,
                                           float Ti, float T, float flo, float fhi, uint32_t)
    {
        const int d = pair_decision(a, P, i, j, r2, Ti, T, flo, fhi);
        own += (uint32_t)(d >> 1);
        if (!(d & 1)) return;
        cnt++;
        density_pair_fp64<KERN, GH>(*pa, xi, yi, zi, w, lz, kn, j, sum, sumd);
    }
};

template <int KERN, bool GH>
struct MomSinkD {
    const PairArgs* pa;
    SideD I;
    int kn;
    uint32_t* q;
    uint32_t head, tail;
    double ax, ay, az, du;

    __device__ __forceinline__ uint32_t mark() const { return 0u; }
    __device__ __forceinline__ void decide(const NbArgs& a, const PatchDev* P, int64_t i, uint32_t j, float r2,
                                           float, float T, float flo, float, uint32_t)
    {
        if (!union_decision(a, P, i, j, r2, T, flo)) return;
        q[32 * (tail & (kQueue - 1))] = j;
        tail++;
    }
    // every queued pair, in order
    __device__ __forceinline__ void group_end(uint32_t)
    {
        for (; head != tail; head++) {
            const PairTermsD t = momentum_pair_fp64<KERN, GH>(*pa, I, q[32 * (head & (kQueue - 1))], kn);
            ax += t.ax;
            ay += t.ay;
            az += t.az;
            du += t.du;
        }
    }
    __device__ __forceinline__ void finish() { group_end(0u); }
};

__device__ __forceinline__ uint32_t fused_warp_sum(uint32_t v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// |N(i)| summed over the warp's particles into the pair counter the lists
// keep (entries listed)
__device__ __forceinline__ void count_pairs(const NbArgs& a, uint32_t cnt)
{
    const uint32_t tot = fused_warp_sum(cnt);
    if ((threadIdx.x & 31) == 0 && tot) atomicAdd(&a.pool_used[1], (unsigned long long)tot);
}

// ---- kernels ----------------------------------------------------------------
template <int K, int KERN, bool GH>
__global__ void __launch_bounds__(32 * kNbtWarps, SPH_FUSED_DEN_MINB)
    k_fused_density_mixed(NbArgs a, const __grid_constant__ PairArgs pa)
{
    if (*a.status & kStBad) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float kb8 = (float)(8.0 * pa.kb), gam = (float)pa.gamma;
    const PairSrc src = pair_src(pa);
    for (int64_t q = (int64_t)blockIdx.x * kNbtWarps + warp; q < a.nunits; q += (int64_t)gridDim.x * kNbtWarps) {
        const WorkItem U = a.units[q];
        const PatchDev* P = a.pd + U.patch;
        const int64_t i = U.begin + lane;
        uint32_t cnt = 0;
        if (i < U.end) {
            const bool big = i >= P->end - (int64_t)P->nbig;
            DensSink<KERN, GH> s = {src, pair_side(pa, P, i), pa.r.rv[i].w, pa.kernel_n, P->zmode,
                                    0.0f, 0.0f, 0.0f, 0.0f, 0u, 0u};
            walk_all<DensSink<KERN, GH>, K>(a, P, i, big, s);
            density_finish<GH>(pa, i, s.I.ri.w, s.inv2h, kb8, gam, s.sum, s.comp, s.sumd, s.compd);
            a.cnt[i] = s.cnt;
            a.nown[i] = s.own;
            cnt = s.cnt;
        }
        count_pairs(a, cnt);
    }
}

template <int K, int KERN, bool GH>
__global__ void __launch_bounds__(32 * kNbtWarps, SPH_FUSED_MOM_MINB)
    k_fused_momentum_mixed(NbArgs a, const __grid_constant__ PairArgs pa)
{
    __shared__ uint32_t qbuf[kNbtWarps * 32 * kQueue];
    if (*a.status & kStBad) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float gscale = (float)KernF<KERN>::grad_scale(pa.kb, pa.kernel_n);
    const MomConst Kc = {0.25f * (float)pa.eps, 0.5f * (float)pa.beta, 0.5f * (float)pa.alpha};
    const PairSrc src = pair_src(pa);
    uint32_t* qlane = qbuf + warp * (32 * kQueue) + lane;
    for (int64_t q = (int64_t)blockIdx.x * kNbtWarps + warp; q < a.nunits; q += (int64_t)gridDim.x * kNbtWarps) {
        const WorkItem U = a.units[q];
        const PatchDev* P = a.pd + U.patch;
        const int64_t i = U.begin + lane;
        if (i < U.end) {
            const bool big = i >= P->end - (int64_t)P->nbig;
            const float4 vi = pa.r.rv[i];
            const float wi2 = vi.w * vi.w;
            MomSink<KERN, GH> s = {src, pair_side(pa, P, i), vi, pa.r.rt[i], wi2 * wi2 * vi.w, Kc,
                                   pa.kernel_n, P->zmode, qlane, 0u, 0u, {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f}};
            walk_all<MomSink<KERN, GH>, K>(a, P, i, big, s);
            s.finish();
            momentum_finish(pa, i, gscale, s.A);
        }
    }
}

template <int K, int KERN, bool GH>
__global__ void __launch_bounds__(32 * kNbtWarps, SPH_FUSED_DEN_MINB)
    k_fused_density_fp64(NbArgs a, const __grid_constant__ PairArgs pa)
{
    if (*a.status & kStBad) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t q = (int64_t)blockIdx.x * kNbtWarps + warp; q < a.nunits; q += (int64_t)gridDim.x * kNbtWarps) {
        const WorkItem U = a.units[q];
        const PatchDev* P = a.pd + U.patch;
        const int64_t i = U.begin + lane;
        uint32_t cnt = 0;
        if (i < U.end) {
            const bool big = i >= P->end - (int64_t)P->nbig;
            DensSinkD<KERN, GH> s = {&pa, pa.s.x[i], pa.s.y[i], pa.s.z[i], pa.f.w[i], P->lz,
                                     pa.kernel_n, 0.0, 0.0, 0u, 0u};
            walk_all<DensSinkD<KERN, GH>, K>(a, P, i, big, s);
            density_finish_fp64<GH>(pa, i, s.sum, s.sumd);
            a.cnt[i] = s.cnt;
            a.nown[i] = s.own;
            cnt = s.cnt;
        }
        count_pairs(a, cnt);
    }
}

template <int K, int KERN, bool GH>
__global__ void __launch_bounds__(32 * kNbtWarps, SPH_FUSED_MOM_MINB)
    k_fused_momentum_fp64(NbArgs a, const __grid_constant__ PairArgs pa)
{
    __shared__ uint32_t qbuf[kNbtWarps * 32 * kQueue];
    if (*a.status & kStBad) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double S80 = KernF<KERN>::grad_scale(pa.kb, pa.kernel_n);
    uint32_t* qlane = qbuf + warp * (32 * kQueue) + lane;
    for (int64_t q = (int64_t)blockIdx.x * kNbtWarps + warp; q < a.nunits; q += (int64_t)gridDim.x * kNbtWarps) {
        const WorkItem U = a.units[q];
        const PatchDev* P = a.pd + U.patch;
        const int64_t i = U.begin + lane;
        if (i < U.end) {
            const bool big = i >= P->end - (int64_t)P->nbig;
            MomSinkD<KERN, GH> s = {&pa, side_fp64(pa, P, i), pa.kernel_n, qlane, 0u, 0u, 0.0, 0.0, 0.0, 0.0};
            walk_all<MomSinkD<KERN, GH>, K>(a, P, i, big, s);
            s.finish();
            momentum_finish_fp64(pa, i, S80, s.ax, s.ay, s.az, s.du);
        }
    }
}

// grid: the resident CTAs of every SM (as the list builder)
template <typename Kern>
void launch_fused(const Launch& L, Kern kern, const NbArgs& a, const PairArgs& pa)
{
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * kNbtWarps, 0);
    if (per_sm < 1) per_sm = 1;
    int64_t blocks = (int64_t)L.sms * per_sm;
    const int64_t need = (a.nunits + kNbtWarps - 1) / kNbtWarps;
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, 32 * kNbtWarps, 0, L.stream>>>(a, pa);
}

#define SPH_FUSED_K(KERNEL, KERN, GH, K, L, a, pa)                                               \
    switch (K) {                                                                                  \
    case 1: launch_fused(L, KERNEL<1, KERN, GH>, a, pa); break;                                   \
    case 2: launch_fused(L, KERNEL<2, KERN, GH>, a, pa); break;                                   \
    default: launch_fused(L, KERNEL<3, KERN, GH>, a, pa); break;                                  \
    }
#define SPH_FUSED_DISPATCH(KERNEL, K, L, a, pa)                                                   \
    if ((pa).kernel == SPH_KERNEL_SINC) {                                                         \
        if ((pa).grad_h) { SPH_FUSED_K(KERNEL, SPH_KERNEL_SINC, true, K, L, a, pa); }             \
        else { SPH_FUSED_K(KERNEL, SPH_KERNEL_SINC, false, K, L, a, pa); }                        \
    } else {                                                                                      \
        if ((pa).grad_h) { SPH_FUSED_K(KERNEL, SPH_KERNEL_WENDLAND, true, K, L, a, pa); }         \
        else { SPH_FUSED_K(KERNEL, SPH_KERNEL_WENDLAND, false, K, L, a, pa); }                    \
    }

}  // namespace sphg
