// sph_sort.cu -- neighbour discovery, first half (Table 1 "Neighbour
// Discovery"; the paper's tree walk is replaced by a Morton-ordered cell
// grid): per-patch bounding box and largest h (FP64, ordered-integer
// atomics), grid parameters, Morton cell keys, a stable LSD radix sort of
// (key, slot), and the gather of every particle field into the sorted order,
// which also writes the cell table and the FP32 cell-relative records.
// Also the device-wide exclusive scan used by the radix sort and the CSR.
#include "sph_internal.cuh"

namespace sphg {

static inline int blocks_for(int64_t work, int threads, int sms, int per_sm)
{
    int64_t b = (work + threads - 1) / threads;
    int64_t cap = (int64_t)sms * per_sm;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

__device__ __forceinline__ unsigned long long umin64(unsigned long long a, unsigned long long b)
{
    return a < b ? a : b;
}
__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b)
{
    return a > b ? a : b;
}

// ---------------------------------------------------------------------------
// A1a: per-patch min/max of x, y and max of h; one block per work item (a
// chunk of one patch), one atomic per block and value.  Min/max are exact,
// so the result does not depend on the order of the atomics.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_reduce_bbox(State s, const WorkItem* items, int nitems,
                                                     PatchRed* red)
{
    __shared__ unsigned long long sh[5][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const WorkItem w = items[it];
        unsigned long long v[5] = {~0ull, ~0ull, 0ull, 0ull, 0ull};
        for (int64_t i = w.begin + threadIdx.x; i < w.end; i += blockDim.x) {
            unsigned long long a = ord_f64(s.x[i]), b = ord_f64(s.y[i]), c = ord_f64(s.h[i]);
            v[0] = umin64(v[0], a);
            v[1] = umin64(v[1], b);
            v[2] = umax64(v[2], a);
            v[3] = umax64(v[3], b);
            v[4] = umax64(v[4], c);
        }
        for (int o = 16; o > 0; o >>= 1) {
            v[0] = umin64(v[0], __shfl_xor_sync(0xffffffffu, v[0], o));
            v[1] = umin64(v[1], __shfl_xor_sync(0xffffffffu, v[1], o));
            v[2] = umax64(v[2], __shfl_xor_sync(0xffffffffu, v[2], o));
            v[3] = umax64(v[3], __shfl_xor_sync(0xffffffffu, v[3], o));
            v[4] = umax64(v[4], __shfl_xor_sync(0xffffffffu, v[4], o));
        }
        if (lane == 0)
            for (int q = 0; q < 5; q++) sh[q][warp] = v[q];
        __syncthreads();
        if (threadIdx.x == 0) {
            const int nw = blockDim.x >> 5;
            for (int ww = 1; ww < nw; ww++) {
                v[0] = umin64(v[0], sh[0][ww]);
                v[1] = umin64(v[1], sh[1][ww]);
                v[2] = umax64(v[2], sh[2][ww]);
                v[3] = umax64(v[3], sh[3][ww]);
                v[4] = umax64(v[4], sh[4][ww]);
            }
            PatchRed* r = red + w.patch;
            atomicMin(&r->xmin, v[0]);
            atomicMin(&r->ymin, v[1]);
            atomicMax(&r->xmax, v[2]);
            atomicMax(&r->ymax, v[3]);
            atomicMax(&r->hmax, v[4]);
        }
        __syncthreads();
    }
}

int launch_reduce_bbox(const Launch& L, const State& s, const WorkItem* items, int nitems,
                       PatchRed* red)
{
    if (nitems <= 0) return 0;
    int grid = nitems < L.sms * 8 ? nitems : L.sms * 8;
    k_reduce_bbox<<<grid, 256, 0, L.stream>>>(s, items, nitems, red);
    return 1;
}

__global__ void k_reset_red(int npatch, PatchRed* red)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < npatch) {
        red[p].xmin = ~0ull;
        red[p].ymin = ~0ull;
        red[p].xmax = 0ull;
        red[p].ymax = 0ull;
        red[p].hmax = 0ull;
        red[p].hcmin = ~0ull;
        for (int b = 0; b < kHBins; b++) red[p].hist[b] = 0u;
    }
}

// ---------------------------------------------------------------------------
// A1a': per patch, a histogram of h / h_max in kHBins bins (integer counts,
// so independent of the order of the atomics); it sets the class threshold.
// Lanes of a warp that fall into the same bin (on a lattice, all of them)
// add their count with one atomic.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_h_hist(State s, const WorkItem* items, int nitems, PatchRed* red)
{
    __shared__ uint32_t hist[kHBins];
    const int lane = threadIdx.x & 31;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const WorkItem w = items[it];
        for (int b = threadIdx.x; b < kHBins; b += blockDim.x) hist[b] = 0u;
        __syncthreads();
        const double hmax = unord_f64(red[w.patch].hmax);
        const double scale = hmax > 0.0 ? (double)kHBins / hmax : 0.0;
        // warp-uniform trip count (blockDim is a multiple of 32)
        for (int64_t i0 = w.begin; i0 < w.end; i0 += blockDim.x) {
            const int64_t i = i0 + threadIdx.x;
            int b = -1;
            if (i < w.end) {
                const double t = s.h[i] * scale;
                b = t >= 0.0 && t < (double)kHBins ? (int)t : kHBins - 1;
            }
            const unsigned peers = __match_any_sync(0xffffffffu, b);
            if (b >= 0 && lane == __ffs(peers) - 1) atomicAdd(&hist[b], (uint32_t)__popc(peers));
        }
        __syncthreads();
        for (int b = threadIdx.x; b < kHBins; b += blockDim.x)
            if (hist[b]) atomicAdd(&red[w.patch].hist[b], hist[b]);
        __syncthreads();
    }
}

int launch_h_hist(const Launch& L, const State& s, const WorkItem* items, int nitems, PatchRed* red)
{
    if (nitems <= 0) return 0;
    int grid = nitems < L.sms * 8 ? nitems : L.sms * 8;
    k_h_hist<<<grid, 256, 0, L.stream>>>(s, items, nitems, red);
    return 1;
}

int launch_reset_red(const Launch& L, int npatch, PatchRed* red)
{
    k_reset_red<<<(npatch + 255) / 256, 256, 0, L.stream>>>(npatch, red);
    return 1;
}

// ---------------------------------------------------------------------------
// A1b: grid of each patch.  Class threshold h_s: the upper edge of the
// lowest histogram bin above which at most 1/kBigShare of the patch lies (h_s
// = h_max, no big particles, when that edge is above 0.8 h_max).  Fine cell
// edge s = 2 h_s cell_factor (with margin), stencil half-extent K = 1 for
// cell_factor >= 1, 2 for >= 1/2, else 3, so K s >= 2 h_s; with K = 3 the
// edge is also at least min(h_s, kCellMed h_median).  Coarse cells are aligned blocks
// of 2^kc fine cells with 2^kc s >= 2 h_max, so the 3 x 3 x 3 coarse block
// around a particle holds every big particle that can reach it.  At most 128
// cells per axis and cell_cap fine + coarse cells per patch (s grows if not).
// Along z: ncz = floor(lz / s) cells of edge lz / ncz; when fewer than 2K+1,
// every z cell is visited once and the minimum image is taken in FP32.
// ---------------------------------------------------------------------------
__global__ void k_grid_params(int npatch, const PatchRed* red, PatchDev* pd, double cell_factor,
                              int* status)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npatch) return;
    PatchDev P = pd[p];
    const int K = stencil_k(cell_factor);
    double xmin = 0, ymin = 0, xmax = 0, ymax = 0, hmax = 0;
    const int64_t np = P.end - P.begin;
    if (np > 0) {
        xmin = unord_f64(red[p].xmin);
        ymin = unord_f64(red[p].ymin);
        xmax = unord_f64(red[p].xmax);
        ymax = unord_f64(red[p].ymax);
        hmax = unord_f64(red[p].hmax);
    }
    double ex = xmax - xmin, ey = ymax - ymin;
    if (!isfinite(ex) || !isfinite(ey) || !isfinite(hmax) || !isfinite(xmin) || !isfinite(ymin)) {
        // non-finite positions: flag, and keep a one-cell grid so that every
        // index computed from it stays inside the cell table
        atomicOr(status, kStNonFinite);
        xmin = ymin = 0.0;
        ex = ey = 0.0;
        hmax = 0.0;
    }
    // class threshold from the histogram of h / h_max
    double hs = hmax;
    {
        const int64_t allow = np / kBigShare;
        int64_t above = 0;
        int b = kHBins - 1;
        while (b > 0 && above + (int64_t)red[p].hist[b] <= allow) {
            above += red[p].hist[b];
            b--;
        }
        const double edge = hmax * (double)(b + 1) / (double)kHBins;
        if (edge < 0.8 * hmax) hs = edge;
    }
    double s = 2.0 * hs * cell_factor * kCellMargin;
    // the median of h, from the histogram, to a bin
    double hmed = hmax;
    {
        int64_t acc = 0;
        for (int b = 0; b < kHBins; b++) {
            acc += red[p].hist[b];
            if (2 * acc >= np) {
                hmed = hmax * ((double)b + 0.5) / (double)kHBins;
                break;
            }
        }
    }
    if (K == 3) {
        // the stencil reaches 3 cells, so cells may be finer than h_s: as
        // fine as 2 h_s cell_factor, but not below min(h_s, kCellMed h_med),
        // the edge that served the interior particles best.  With a narrow
        // spread of h this is the h_s-sized cell of cell_factor 1/2.
        const double sm = fmin(hs, kCellMed * hmed) * kCellMargin;
        if (s < sm) s = sm;
    }
    const double sext = fmax(ex, ey) / (double)(kMaxCellsAxis - 1) * kCellMargin;
    if (s < sext) s = sext;
    if (!(s > 0.0)) s = P.lz > 0.0 ? P.lz : 1.0;
    int64_t ncx = 1, ncy = 1, ncz = 1, ncxc = 1, ncyc = 1, nczc = 1;
    int kc = 0;
    bool fits = false;
    for (int iter = 0; iter < 200 && !fits; iter++) {
        ncx = (int64_t)floor(ex / s) + 1;
        ncy = (int64_t)floor(ey / s) + 1;
        ncz = (int64_t)floor(P.lz / s);
        if (ncz < 1) ncz = 1;
        if (ncz > kMaxCellsAxis) ncz = kMaxCellsAxis;
        kc = 0;
        if (hs < hmax) {
            while (kc < kMortonBits && (double)(1 << kc) * s < 2.0 * hmax * kCellMargin) kc++;
            // whole coarse cells along the period (a partial one would let a big
            // particle two coarse cells away across the wrap reach the block)
            if (ncz >= (1 << kc)) ncz = (ncz >> kc) << kc;
        } else {
            kc = kMortonBits;   // no big particles: one (empty) coarse cell
        }
        ncxc = (ncx + (1 << kc) - 1) >> kc;
        ncyc = (ncy + (1 << kc) - 1) >> kc;
        nczc = (ncz + (1 << kc) - 1) >> kc;
        fits = ncx <= kMaxCellsAxis && ncy <= kMaxCellsAxis && ncx * ncy * ncz + ncxc * ncyc * nczc <= P.cell_cap;
        if (!fits) s *= 1.25;
    }
    if (!fits || ncx < 1 || ncy < 1) {
        atomicOr(status, kStNonFinite);
        ncx = ncy = ncz = ncxc = ncyc = nczc = 1;
        kc = 0;
    }
    P.xmin = xmin;
    P.ymin = ymin;
    P.hmax = hmax;
    P.s = s;
    P.sz = P.lz / (double)ncz;
    P.ncx = (int)ncx;
    P.ncy = (int)ncy;
    P.ncz = (int)ncz;
    P.K = K;
    P.zmode = ncz >= 2 * K + 1 ? 0 : 1;
    P.s_f = (float)s;
    P.sz_f = (float)P.sz;
    P.lz_f = (float)P.lz;
    P.inv_s_f = (float)(1.0 / s);
    P.inv_sz_f = (float)(1.0 / P.sz);
    P.hmax_f = (float)hmax;
    P.hs = hs;
    P.hs_f = (float)hs;
    P.hmed = hmed;
    P.nbig = 0;
    P.kc = kc;
    P.ncxc = (int)ncxc;
    P.ncyc = (int)ncyc;
    P.nczc = (int)nczc;
    P.zmode_c = nczc >= 3 ? 0 : 1;
    P.coarse_base = P.cell_base + ncx * ncy * ncz;
    pd[p] = P;
}

int launch_grid_params(const Launch& L, int npatch, const PatchRed* red, PatchDev* pd,
                       double cell_factor, int* status)
{
    k_grid_params<<<(npatch + 127) / 128, 128, 0, L.stream>>>(npatch, red, pd, cell_factor, status);
    return 1;
}

// ---------------------------------------------------------------------------
// A1c: key = patch << 22 | big << 21 | Morton(cx, cy, cz), big = (h > h_s),
// cell coordinates in FP32 from the FP64 offset to the grid origin (error <
// 1e-4 cell, inside the margin).  Counts the big particles of each patch.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_keys(int64_t n, State s, const uint16_t* patch_of,
                                              PatchDev* pd, uint32_t* keys, uint32_t* vals)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int p = patch_of[i];
        PatchDev* P = pd + p;
        const bool big = s.h[i] > P->hs;
        // one atomic per warp and patch: the lanes of a warp that share the
        // patch add their big particles together
        const unsigned act = __activemask();
        const unsigned peers = __match_any_sync(act, p);
        const unsigned bigs = __ballot_sync(act, big) & peers;
        if (bigs && (int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&P->nbig, __popc(bigs));
        const float tx = (float)(s.x[i] - P->xmin) * P->inv_s_f;
        const float ty = (float)(s.y[i] - P->ymin) * P->inv_s_f;
        const float tz = (float)(s.z[i] + 0.5 * P->lz) * P->inv_sz_f;
        int cx = (int)floorf(tx), cy = (int)floorf(ty), cz = (int)floorf(tz);
        cx = min(max(cx, 0), P->ncx - 1);
        cy = min(max(cy, 0), P->ncy - 1);
        cz = min(max(cz, 0), P->ncz - 1);
        keys[i] = ((uint32_t)p << kPatchShift) | ((uint32_t)big << kClassShift) | part1by2((uint32_t)cx) |
                  (part1by2((uint32_t)cy) << 1) | (part1by2((uint32_t)cz) << 2);
        vals[i] = (uint32_t)i;
    }
}

int launch_keys(const Launch& L, int64_t n, const State& s, const uint16_t* patch_of,
                PatchDev* pd, uint32_t* keys, uint32_t* vals)
{
    if (n <= 0) return 0;
    k_keys<<<blocks_for(n, 256, L.sms, 16), 256, 0, L.stream>>>(n, s, patch_of, pd, keys, vals);
    return 1;
}

// ---------------------------------------------------------------------------
// Block-wide exclusive scan helpers (blockDim.x a multiple of 32, <= 1024).
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v)
{
    const int lane = threadIdx.x & 31;
    for (int o = 1; o < 32; o <<= 1) {
        T t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// returns the exclusive prefix of v over the block; *total receives the sum
template <typename T>
__device__ __forceinline__ T block_excl_scan(T v, T* total, T* sh /* >= 33 */)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T inc = warp_incl_scan(v);
    if (lane == 31) sh[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T w = lane < nw ? sh[lane] : T(0);
        T wi = warp_incl_scan(w);
        if (lane < nw) sh[lane] = wi - w;
        if (lane == 31) sh[32] = wi;
    }
    __syncthreads();
    T res = inc - v + sh[warp];
    *total = sh[32];
    __syncthreads();
    return res;
}

// ---------------------------------------------------------------------------
// Device-wide exclusive scan, reduce-then-scan in three launches.
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

template <typename Tin, typename Tout>
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const Tin* in, int64_t n, Tout* part)
{
    __shared__ Tout sh[33];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    Tout v = 0;
    for (int k = 0; k < kScanItems; k++) {
        int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
        if (i < n) v += (Tout)in[i];
    }
    Tout tot;
    block_excl_scan<Tout>(v, &tot, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

template <typename Tout>
__global__ void __launch_bounds__(1024) k_scan_spine(Tout* part, int64_t nb)
{
    __shared__ Tout sh[33];
    Tout carry = 0;
    for (int64_t base = 0; base < nb; base += blockDim.x) {
        int64_t i = base + threadIdx.x;
        Tout v = i < nb ? part[i] : Tout(0);
        Tout tot;
        Tout ex = block_excl_scan<Tout>(v, &tot, sh);
        if (i < nb) part[i] = ex + carry;
        carry += tot;
    }
}

template <typename Tin, typename Tout>
__global__ void __launch_bounds__(kScanThreads) k_scan_down(const Tin* in, int64_t n, const Tout* part,
                                                           Tout* out, int write_total)
{
    __shared__ Tout sh[33];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    Tout loc[kScanItems];
    Tout sum = 0;
    for (int k = 0; k < kScanItems; k++) {
        int64_t i = base + k;
        Tout v = i < n ? (Tout)in[i] : Tout(0);
        loc[k] = sum;
        sum += v;
    }
    Tout tot;
    Tout ex = block_excl_scan<Tout>(sum, &tot, sh) + part[blockIdx.x];
    for (int k = 0; k < kScanItems; k++) {
        int64_t i = base + k;
        if (i < n) out[i] = ex + loc[k];
    }
    if (write_total && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = part[blockIdx.x] + tot;
}

int64_t scan_tmp_words(int64_t n) { return (n + kScanTile - 1) / kScanTile + 1; }

int launch_scan_u32_to_u64(const Launch& L, int64_t n, const uint32_t* in, uint64_t* out, uint64_t* tmp)
{
    if (n <= 0) {
        cudaMemsetAsync(out, 0, sizeof(uint64_t), L.stream);
        return 0;
    }
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    k_scan_reduce<uint32_t, uint64_t><<<(unsigned)nb, kScanThreads, 0, L.stream>>>(in, n, tmp);
    k_scan_spine<uint64_t><<<1, 1024, 0, L.stream>>>(tmp, nb);
    k_scan_down<uint32_t, uint64_t><<<(unsigned)nb, kScanThreads, 0, L.stream>>>(in, n, tmp, out, 1);
    return 3;
}

static int scan_u32(const Launch& L, int64_t n, const uint32_t* in, uint32_t* out, uint32_t* tmp)
{
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    k_scan_reduce<uint32_t, uint32_t><<<(unsigned)nb, kScanThreads, 0, L.stream>>>(in, n, tmp);
    k_scan_spine<uint32_t><<<1, 1024, 0, L.stream>>>(tmp, nb);
    k_scan_down<uint32_t, uint32_t><<<(unsigned)nb, kScanThreads, 0, L.stream>>>(in, n, tmp, out, 0);
    return 3;
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort, 8-bit digits.  Per pass: a digit histogram per
// tile of 4096 keys (digit-major), an exclusive scan of the histograms, and a
// scatter that ranks keys stably inside the tile (warp match + per-warp
// counters, warps in tile order), stages the tile in shared memory in digit
// order and writes each digit run contiguously.
// ---------------------------------------------------------------------------
constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsStrips = 16;
constexpr int kRsTile = kRsWarps * 32 * kRsStrips;  // 4096

__global__ void __launch_bounds__(kRsThreads) k_rs_hist(const uint32_t* keys, int64_t n, int shift,
                                                       uint32_t* hist, int ntiles)
{
    __shared__ uint32_t sh[256];
    const int lane = threadIdx.x & 31;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        sh[threadIdx.x] = 0;
        __syncthreads();
        const int64_t base = (int64_t)tile * kRsTile;
        for (int k = threadIdx.x; k < kRsTile; k += blockDim.x) {
            const int64_t i = base + k;
            const uint32_t d = i < n ? ((keys[i] >> shift) & 255u) : 256u;
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            if (d < 256u && lane == __ffs(peers) - 1) atomicAdd(&sh[d], (uint32_t)__popc(peers));
        }
        __syncthreads();
        hist[(int64_t)threadIdx.x * ntiles + tile] = sh[threadIdx.x];
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kRsThreads) k_rs_scatter(const uint32_t* kin, const uint32_t* vin,
                                                          int64_t n, int shift, const uint32_t* hoff,
                                                          int ntiles, uint32_t* kout, uint32_t* vout)
{
    __shared__ uint32_t s_keys[kRsTile];
    __shared__ uint32_t s_vals[kRsTile];
    __shared__ uint32_t s_wcnt[kRsWarps][256];
    __shared__ uint32_t s_dstart[256];
    __shared__ uint32_t s_goff[256];
    __shared__ uint32_t s_scan[33];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        for (int k = threadIdx.x; k < kRsWarps * 256; k += blockDim.x) (&s_wcnt[0][0])[k] = 0;
        __syncthreads();
        uint32_t kr[kRsStrips], vr[kRsStrips];
        uint16_t pr[kRsStrips];
        const int64_t wbase = (int64_t)tile * kRsTile + (int64_t)warp * 32 * kRsStrips;
#pragma unroll
        for (int t = 0; t < kRsStrips; t++) {
            const int64_t i = wbase + t * 32 + lane;
            const bool valid = i < n;
            const uint32_t key = valid ? kin[i] : 0xffffffffu;
            const uint32_t val = valid ? vin[i] : 0u;
            const uint32_t d = valid ? ((key >> shift) & 255u) : 256u;
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            const int rank = __popc(peers & ((1u << lane) - 1u));
            uint32_t before = 0;
            if (valid) before = s_wcnt[warp][d];
            __syncwarp();
            if (valid && lane == __ffs(peers) - 1) s_wcnt[warp][d] = before + (uint32_t)__popc(peers);
            __syncwarp();
            kr[t] = key;
            vr[t] = val;
            pr[t] = (uint16_t)(before + rank);
        }
        __syncthreads();
        {   // per digit: exclusive offsets of the warps, then digit starts in the tile
            const int d = threadIdx.x;
            uint32_t run = 0;
            for (int w = 0; w < kRsWarps; w++) {
                uint32_t c = s_wcnt[w][d];
                s_wcnt[w][d] = run;
                run += c;
            }
            uint32_t tot;
            s_dstart[d] = block_excl_scan<uint32_t>(run, &tot, s_scan);
            s_goff[d] = hoff[(int64_t)d * ntiles + tile];
        }
        __syncthreads();
#pragma unroll
        for (int t = 0; t < kRsStrips; t++) {
            const int64_t i = wbase + t * 32 + lane;
            if (i < n) {
                const uint32_t d = (kr[t] >> shift) & 255u;
                const uint32_t lp = s_dstart[d] + s_wcnt[warp][d] + pr[t];
                s_keys[lp] = kr[t];
                s_vals[lp] = vr[t];
            }
        }
        __syncthreads();
        const int64_t rem = n - (int64_t)tile * kRsTile;
        const int tn = rem < kRsTile ? (int)rem : kRsTile;
        for (int k = threadIdx.x; k < tn; k += blockDim.x) {
            const uint32_t key = s_keys[k];
            const uint32_t d = (key >> shift) & 255u;
            const uint32_t g = s_goff[d] + ((uint32_t)k - s_dstart[d]);
            kout[g] = key;
            vout[g] = s_vals[k];
        }
        __syncthreads();
    }
}

size_t radix_hist_words(int64_t n)
{
    int64_t ntiles = (n + kRsTile - 1) / kRsTile;
    if (ntiles < 1) ntiles = 1;
    return (size_t)(256 * ntiles);
}

int launch_radix_sort(const Launch& L, int64_t n, int passes, uint32_t* keys, uint32_t* vals,
                      uint32_t* keys_alt, uint32_t* vals_alt, uint32_t* hist, uint32_t* scan_tmp)
{
    if (n <= 1) return 0;
    const int ntiles = (int)((n + kRsTile - 1) / kRsTile);
    const int grid = ntiles < L.sms * 4 ? ntiles : L.sms * 4;
    const int64_t nh = (int64_t)256 * ntiles;
    int launches = 0;
    uint32_t *ki = keys, *vi = vals, *ko = keys_alt, *vo = vals_alt;
    for (int ps = 0; ps < passes; ps++) {
        const int shift = 8 * ps;
        k_rs_hist<<<grid, kRsThreads, 0, L.stream>>>(ki, n, shift, hist, ntiles);
        launches += 1 + scan_u32(L, nh, hist, hist, scan_tmp);
        k_rs_scatter<<<grid, kRsThreads, 0, L.stream>>>(ki, vi, n, shift, hist, ntiles, ko, vo);
        launches++;
        uint32_t* t = ki; ki = ko; ko = t;
        t = vi; vi = vo; vo = t;
    }
    if (ki != keys) {   // odd number of passes: copy back
        cudaMemcpyAsync(keys, ki, (size_t)n * 4, cudaMemcpyDeviceToDevice, L.stream);
        cudaMemcpyAsync(vals, vi, (size_t)n * 4, cudaMemcpyDeviceToDevice, L.stream);
    }
    return launches;
}

// ---------------------------------------------------------------------------
// Row-length bins of the pair sums: key = octave of |N(i)|, sorted stably by
// one radix pass; the bin starts are the scanned digit offsets of the first
// tile.
// ---------------------------------------------------------------------------
__global__ void k_octave_keys(int64_t n, const uint32_t* cnt, uint32_t* keys, uint32_t* vals)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t c = cnt[i];
        // 0 for an empty row, else 1 + ceil(log2 c) (32 - clz(c - 1) = ceil(log2 c))
        const int o = c == 0u ? 0 : 33 - __clz(c - 1u);
        keys[i] = (uint32_t)min(o, kPairOctaves - 1);
        vals[i] = (uint32_t)i;
    }
}

__global__ void k_octave_bounds(const uint32_t* hist, int ntiles, int64_t n, uint32_t* bounds)
{
    const int o = threadIdx.x;
    if (o < kPairOctaves) bounds[o] = hist[(int64_t)o * ntiles];
    if (o == kPairOctaves) bounds[o] = (uint32_t)n;
}

int launch_pair_bins(const Launch& L, int64_t n, const uint32_t* cnt, uint32_t* keys, uint32_t* order,
                     uint32_t* keys_alt, uint32_t* vals_alt, uint32_t* hist, uint32_t* scan_tmp, uint32_t* bounds)
{
    if (n <= 0) return 0;
    int64_t blocks = (n + 255) / 256;
    if (blocks > (int64_t)L.sms * 16) blocks = (int64_t)L.sms * 16;
    k_octave_keys<<<(unsigned)blocks, 256, 0, L.stream>>>(n, cnt, keys, order);
    int launches = 1;
    const int ntiles = (int)((n + kRsTile - 1) / kRsTile);
    if (n > 1) {
        launches += launch_radix_sort(L, n, 1, keys, order, keys_alt, vals_alt, hist, scan_tmp);
    } else {
        // one particle, no sort: every bound but the last is 0, so it is
        // summed by the last octave's launch (any lanes-per-particle count
        // gives a correct sum)
        cudaMemsetAsync(hist, 0, sizeof(uint32_t) * 256, L.stream);
    }
    k_octave_bounds<<<1, 32, 0, L.stream>>>(hist, ntiles, n, bounds);
    return launches + 1;
}

// ---------------------------------------------------------------------------
// Gather every field into sorted order, write the permutation, the
// cell table (start/end by key boundaries, largest h per cell) and the FP32
// records with positions relative to the particle's cell origin.  Also forms
// the time-centred velocity v_{n-1/2} + a_{n-1} dt_{n-1}/2 used by the
// viscosity and the energy equation.
// ---------------------------------------------------------------------------
// the FP32 records of sorted slot k in cell (cx, cy, cz) of patch P: offsets
// from the cell origin, 4 hq^2 (hq: the h of the search), and for
// the pair sums the mass, the time-centred velocity v + a_{n-1} dt_{n-1}/2
// and 1/(2h) (mixed), or the same in FP64.  The z offset is taken from the
// image of z nearest the cell's centre: a particle that has left its cell
// since the sort (reused lists) may have crossed the periodic z boundary, and
// the pair separation, which wraps at most once, needs every offset within
// about a cell of its cell.  A particle inside its cell is its own nearest
// image, so this changes nothing right after a sort.
__device__ __forceinline__ void write_records(int64_t k, const PatchDev* P, uint32_t cx, uint32_t cy, uint32_t cz,
                                              double x, double y, double z, double vx, double vy, double vz,
                                              double m, double h, double u, double axp, double ayp, double azp,
                                              float hq, Recs& r, Fp64& f, int mixed)
{
    const float ox = (float)(x - (P->xmin + (double)cx * P->s));
    const float oy = (float)(y - (P->ymin + (double)cy * P->s));
    double ozd = z - (-0.5 * P->lz + (double)cz * P->sz);
    const double oc = ozd - 0.5 * P->sz;
    if (oc > 0.5 * P->lz) ozd -= P->lz;
    else if (oc < -0.5 * P->lz) ozd += P->lz;
    const float oz = (float)ozd;
    const float hf = (float)h;
    r.r4[k] = make_float4(ox, oy, oz, 4.0f * hq * hq);
    const double half = P->step > 0 ? 0.5 * P->dt_prev : 0.0;
    const double vhx = vx + axp * half, vhy = vy + ayp * half, vhz = vz + azp * half;
    if (mixed) {
        r.r5[k] = make_float4(ox, oy, oz, (float)m);
        r.rv[k] = make_float4((float)vhx, (float)vhy, (float)vhz, 0.5f / hf);
        r.uf[k] = (float)u;
    } else {
        f.vhx[k] = vhx;
        f.vhy[k] = vhy;
        f.vhz[k] = vhz;
        const double w = 0.5 / h;
        f.w[k] = w;
        f.w5[k] = w * w * w * w * w;
    }
}

__global__ void __launch_bounds__(256) k_gather(int64_t n, const uint32_t* skeys, const uint32_t* svals,
                                                State src, State dst, const uint32_t* perm_src,
                                                uint32_t* perm_dst, const PatchDev* pd, Grid g,
                                                Recs r, Fp64 f, int mixed, RowHint hint,
                                                const double* hsearch, double* hsearch_out)
{
    const bool have_hint = *hint.valid != 0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t key = skeys[k];
        const uint32_t si = svals[k];
        const PatchDev* P = pd + (key >> kPatchShift);
        const double x = src.x[si], y = src.y[si], z = src.z[si];
        const double vx = src.vx[si], vy = src.vy[si], vz = src.vz[si];
        const double m = src.m[si], h = src.h[si];
        const double axp = src.axp[si], ayp = src.ayp[si], azp = src.azp[si];
        dst.x[k] = x; dst.y[k] = y; dst.z[k] = z;
        dst.vx[k] = vx; dst.vy[k] = vy; dst.vz[k] = vz;
        dst.m[k] = m; dst.h[k] = h;
        dst.u[k] = src.u[si];
        dst.du_prev[k] = src.du_prev[si];
        dst.axp[k] = axp; dst.ayp[k] = ayp; dst.azp[k] = azp;
        perm_dst[k] = perm_src[si];
        hint.rowcap[k] = have_hint ? hint.cnt_prev[si] : kNoHint;

        const uint32_t mort = key & kMortonMask;
        const bool big = (key >> kClassShift) & 1u;
        const uint32_t cx = compact1by2(mort), cy = compact1by2(mort >> 1), cz = compact1by2(mort >> 2);
        g.cellxyz[k] = cx | (cy << 8) | (cz << 16);
        // h of the search
        const float hf = (float)(hsearch ? hsearch[si] : h);
        if (hsearch_out) hsearch_out[k] = hsearch[si];
        write_records(k, P, cx, cy, cz, x, y, z, vx, vy, vz, m, h, dst.u[k], axp, ayp, azp, hf, r, f, mixed);
        if (!big) {
            // fine cell of small particles: bounded by a change of key
            const int64_t lin = P->cell_base + ((int64_t)cz * P->ncy + cy) * P->ncx + cx;
            if (k == P->begin || skeys[k - 1] != key) g.cell[lin].x = (uint32_t)k;
            if (k + 1 == P->end || skeys[k + 1] != key) g.cell[lin].y = (uint32_t)(k + 1);
            atomicMax(&g.cell[lin].z, __float_as_uint(hf));
        } else {
            // coarse cell of big particles: an aligned block of 2^kc fine cells,
            // contiguous in Morton order, bounded by a change of key >> 3 kc
            const int kc = P->kc;
            const int64_t lin = P->coarse_base +
                                ((int64_t)(cz >> kc) * P->ncyc + (cy >> kc)) * P->ncxc + (cx >> kc);
            const uint32_t pre = key >> (3 * kc);
            if (k == P->begin || (skeys[k - 1] >> (3 * kc)) != pre) g.cell[lin].x = (uint32_t)k;
            if (k + 1 == P->end || (skeys[k + 1] >> (3 * kc)) != pre) g.cell[lin].y = (uint32_t)(k + 1);
            atomicMax(&g.cell[lin].z, __float_as_uint(hf));
        }
    }
}

int launch_gather(const Launch& L, int64_t n, const uint32_t* skeys, const uint32_t* svals,
                  const State& src, const State& dst, const uint32_t* perm_src, uint32_t* perm_dst,
                  const PatchDev* pd, const Grid& g, const Recs& r, const Fp64& f, int mixed,
                  const RowHint& hint, const double* hsearch, double* hsearch_out)
{
    if (n <= 0) return 0;
    k_gather<<<blocks_for(n, 256, L.sms, 16), 256, 0, L.stream>>>(n, skeys, svals, src, dst, perm_src,
                                                                 perm_dst, pd, g, r, f, mixed, hint, hsearch,
                                                                 hsearch_out);
    return 1;
}

// records of the current state without a sort (between rebuilds of a reused
// candidate superset): the grid and cells of the last sort, the current
// positions, h and time state
__global__ void __launch_bounds__(256) k_refresh_records(int64_t n, State s, const uint16_t* patch_of,
                                                         const PatchDev* pd, const uint32_t* cellxyz, Recs r,
                                                         Fp64 f, int mixed)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const PatchDev* P = pd + patch_of[k];
        const uint32_t c = cellxyz[k];
        const double h = s.h[k];
        write_records(k, P, c & 255u, (c >> 8) & 255u, c >> 16, s.x[k], s.y[k], s.z[k], s.vx[k], s.vy[k], s.vz[k],
                      s.m[k], h, s.u[k], s.axp[k], s.ayp[k], s.azp[k], (float)h, r, f, mixed);
    }
}

int launch_refresh_records(const Launch& L, int64_t n, const State& s, const uint16_t* patch_of,
                           const PatchDev* pd, const uint32_t* cellxyz, const Recs& r, const Fp64& f, int mixed)
{
    if (n <= 0) return 0;
    k_refresh_records<<<blocks_for(n, 256, L.sms, 16), 256, 0, L.stream>>>(n, s, patch_of, pd, cellxyz, r, f,
                                                                          mixed);
    return 1;
}

// ---------------------------------------------------------------------------
// The tight box of each non-empty fine cell, from its particles' FP32
// offsets, quantised outward to 1/kBoxQ of the cell edge (see Grid).  One
// thread per cell; blockIdx.y is the patch.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int box_q(float o, float inv_edge)
{
    const int q = (int)floorf(o * inv_edge * (float)kBoxQ);
    return min(max(q, 0), kBoxQ - 1);
}

__global__ void __launch_bounds__(256) k_cell_boxes(const PatchDev* pd, Grid g, const float4* r4)
{
    const PatchDev* P = pd + blockIdx.y;
    const int64_t nfine = (int64_t)P->ncx * P->ncy * P->ncz;
    const float inv_s = P->inv_s_f, inv_sz = P->inv_sz_f;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nfine; c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t lin = P->cell_base + c;
        const uint32_t b = g.cell[lin].x, e = g.cell[lin].y;
        if (b >= e) continue;
        int lx = kBoxQ, ly = kBoxQ, lz = kBoxQ, hx = 0, hy = 0, hz = 0;
        for (uint32_t k = b; k < e; k++) {
            const float4 q = r4[k];
            const int qx = box_q(q.x, inv_s), qy = box_q(q.y, inv_s), qz = box_q(q.z, inv_sz);
            lx = min(lx, qx);
            ly = min(ly, qy);
            lz = min(lz, qz);
            hx = max(hx, qx + 1);
            hy = max(hy, qy + 1);
            hz = max(hz, qz + 1);
        }
        g.cell[lin].w = (uint32_t)lx | ((uint32_t)(kBoxQ - hx) << 5) | ((uint32_t)ly << 10) |
                        ((uint32_t)(kBoxQ - hy) << 15) | ((uint32_t)lz << 20) | ((uint32_t)(kBoxQ - hz) << 25);
    }
}

// The largest h within K fine cells of each fine cell along each axis, a
// separable maximum in three passes: along x and along y (in range), then
// over 2K+1 z planes (periodic; with fewer z cells than that, every plane).
// A small particle's search from this cell reaches no farther than
// 2 max(h_i, hnb).  axis 0 reads the cell table's h_max, the others the
// previous pass.
__global__ void __launch_bounds__(256) k_hnb_pass(const PatchDev* pd, Grid g, int K, int axis, const float* in,
                                                  float* out)
{
    const PatchDev* P = pd + blockIdx.y;
    const int ncx = P->ncx, ncy = P->ncy, ncz = P->ncz;
    const int64_t nxy = (int64_t)ncx * ncy;
    const int64_t nfine = nxy * ncz;
    const int n = axis == 0 ? ncx : (axis == 1 ? ncy : ncz);
    const int64_t stride = axis == 0 ? 1 : (axis == 1 ? ncx : nxy);
    // every z plane when they are fewer than 2K+1
    const int kk = axis == 2 && 2 * K + 1 > ncz ? (ncz - 1) / 2 + 1 : K;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nfine; c += (int64_t)gridDim.x * blockDim.x) {
        const int pos = (int)((c / stride) % n);
        const int64_t c0 = c - (int64_t)pos * stride;
        float m = 0.0f;
        for (int d = -kk; d <= kk; d++) {
            int q = pos + d;
            if (axis == 2) q = ((q % n) + n) % n;
            else if (q < 0 || q >= n) continue;
            const int64_t cell = P->cell_base + c0 + (int64_t)q * stride;
            m = fmaxf(m, axis == 0 ? __uint_as_float(g.cell[cell].z) : in[cell]);
        }
        out[P->cell_base + c] = m;
    }
}

int launch_cell_hnb(const Launch& L, int npatch, const PatchDev* pd, const Grid& g, int K, float* tmp)
{
    if (npatch <= 0) return 0;
    const dim3 grid(npatch > 8 ? 8 : (L.sms * 4 + npatch - 1) / npatch, npatch);
    k_hnb_pass<<<grid, 256, 0, L.stream>>>(pd, g, K, 0, nullptr, g.hnb);
    k_hnb_pass<<<grid, 256, 0, L.stream>>>(pd, g, K, 1, g.hnb, tmp);
    k_hnb_pass<<<grid, 256, 0, L.stream>>>(pd, g, K, 2, tmp, g.hnb);
    return 3;
}

// The vote of the cell grid for the next sort: the fine cells that hold
// particles, and among them, in a patch whose spread of h is wide (h_s >
// 1.4 h_median), those whose particles' neighbourhoods have no h above 0.8
// h_s.  Many such cells (h wide but smooth in space, as behind the free
// surface of a patch) favour a 3-cell stencil over median-sized cells; few
// (h varying from particle to particle) favour cells of edge h_s.
__global__ void __launch_bounds__(256) k_cell_vote(const PatchDev* pd, Grid g, unsigned long long* vote)
{
    const PatchDev* P = pd + blockIdx.y;
    const int64_t nfine = (int64_t)P->ncx * P->ncy * P->ncz;
    const bool wide = P->hs > 1.4 * P->hmed;
    const float lim = 0.8f * P->hs_f;
    uint32_t ne = 0, nn = 0;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nfine; c += (int64_t)gridDim.x * blockDim.x) {
        const uint4 cr = g.cell[P->cell_base + c];
        if (cr.x >= cr.y) continue;
        ne++;
        nn += (uint32_t)(wide && g.hnb[P->cell_base + c] < lim);
    }
    for (int o = 16; o > 0; o >>= 1) {
        ne += __shfl_xor_sync(0xffffffffu, ne, o);
        nn += __shfl_xor_sync(0xffffffffu, nn, o);
    }
    if ((threadIdx.x & 31) == 0 && ne) {
        atomicAdd(&vote[0], (unsigned long long)ne);
        atomicAdd(&vote[1], (unsigned long long)nn);
    }
}

int launch_cell_vote(const Launch& L, int npatch, const PatchDev* pd, const Grid& g, unsigned long long* vote)
{
    cudaMemsetAsync(vote, 0, 2 * sizeof(unsigned long long), L.stream);
    if (npatch <= 0) return 0;
    const dim3 grid(npatch > 8 ? 8 : (L.sms * 4 + npatch - 1) / npatch, npatch);
    k_cell_vote<<<grid, 256, 0, L.stream>>>(pd, g, vote);
    return 1;
}

int launch_cell_boxes(const Launch& L, int npatch, const PatchDev* pd, const Grid& g, const float4* r4)
{
    if (npatch <= 0) return 0;
    const int bx = npatch > 8 ? 8 : (L.sms * 4 + npatch - 1) / npatch;
    k_cell_boxes<<<dim3((unsigned)bx, (unsigned)npatch), 256, 0, L.stream>>>(pd, g, r4);
    return 1;
}

}  // namespace sphg
