// sph_internal.cuh -- device data layout and launch declarations shared by
// the CUDA translation units of libsph_gb300.so.  Not part of the C ABI.
//
// Particles live in HBM as structure-of-arrays, sorted by (patch, class,
// Morton cell).  Per patch, the particles with h <= h_s are "small" and the
// few above are "big" (h_s: a high quantile of h, so that about 1/64 of the
// patch is big).  A uniform grid of cells with edge s >= 2 h_s cell_factor
// covers the bounding box in x, y and the period lz in z; a small particle
// searches the (2K+1)^3 cells around its own (K = 1 for cell_factor >= 1,
// 2 for >= 1/2, 3 below) for small neighbours, pruned by the largest h
// around its cell and by each cell's own largest h.  Big
// particles are indexed separately by coarse cells (aligned blocks of 2^kc
// fine cells with edge >= 2 h_max), which every particle searches for big
// neighbours; a big particle searches the fine grid as far as its own 2 h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "../../include/sph.h"

namespace sphg {

constexpr int kMortonBits = 7;                 // per axis: at most 128 cells
constexpr int kMaxCellsAxis = 1 << kMortonBits;
constexpr int kClassShift = 3 * kMortonBits;   // key = patch << 22 | big << 21 | morton
constexpr int kPatchShift = kClassShift + 1;
constexpr uint32_t kMortonMask = (1u << kClassShift) - 1u;
constexpr int kColBits = 25;                   // packed column: j | stencil << 25
constexpr uint32_t kColMask = (1u << kColBits) - 1u;
constexpr int64_t kMaxParticles = int64_t(1) << kColBits;
constexpr int kMaxPatches = 256;
constexpr int kItemChunk = 4096;               // particles per work item
constexpr uint32_t kFarCode = 127;             // column stencil code: offset from the cell coordinates
#ifndef SPH_BIG_SHARE
#define SPH_BIG_SHARE 64
#endif
constexpr int kBigShare = SPH_BIG_SHARE;       // about 1/kBigShare of a patch is big
constexpr int kHFacN = 4096;                   // entries of the h-adaptation factor table

// status word bits (device, sticky until the host clears it)
constexpr int kStOverflow = 1;
constexpr int kStNonFinite = 2;
constexpr int kStTimeout = 4;
constexpr int kStBad = kStOverflow | kStNonFinite | kStTimeout;  // later phases skip

// Guard band of the FP32 neighbour pre-filter: a candidate is decided in FP32
// only when r^2 is outside [T (1 - tol), T (1 + tol)], T the FP64 threshold;
// otherwise the exact FP64 predicate decides.  tol = 2^-13 + 2^-16 s/h_i
// bounds the FP32 rounding of r^2 computed from cell-relative coordinates
// shifted by at most 3 cells (error below 60 * 2^-24 s/h relative to T) with
// a margin of more than 4x.
constexpr float kTolBase = 1.0f / 8192.0f;
constexpr float kTolCell = 1.0f / 65536.0f;
// stencil half-extent for a cell factor: K s >= 2 h_s needs K cell_factor >= 1
__host__ __device__ __forceinline__ int stencil_k(double cell_factor)
{
    return cell_factor >= 1.0 ? 1 : (cell_factor >= 0.5 ? 2 : 3);
}
// Cell edges carry a relative margin so that FP32 cell assignment can never
// separate two particles closer than 2 h_max by more than K cells.
constexpr double kCellMargin = 1.0 + 1.0 / 1024.0;
// with a 3-cell stencil, cells no finer than min(h_s, kCellMed h_median)
constexpr double kCellMed = 1.3;

struct PatchDev {
    int64_t begin, end;          // sorted slot range (fixed after set_patches)
    int64_t cell_base, cell_cap; // slice of the cell tables
    int32_t item_begin, item_end;  // work items of this patch
    double xmin, ymin, s, sz, hmax, lz;
    float s_f, sz_f, lz_f, inv_s_f, inv_sz_f, hmax_f;
    int32_t ncx, ncy, ncz, K;
    int32_t zmode;               // 0: 2K+1 distinct z cells; 1: all z cells + float wrap
    int32_t nbig;                // big particles (h > hs), counted by the key kernel
    double hs;                   // class threshold: small iff h <= hs
    float hs_f;
    double hmed;                 // median of h (histogram bin centre)
    int32_t kc;                  // coarse cell = 2^kc fine cells per axis
    int32_t ncxc, ncyc, nczc;    // coarse grid
    int32_t zmode_c;             // 0: 3 distinct coarse z cells; 1: all of them
    int64_t coarse_base;         // first coarse cell in the cell tables
    // time state
    double dt, dt_prev;
    int64_t step;
};

// Per-patch reduction slots, ordered-integer encoded doubles.
constexpr int kHBins = 64;       // histogram of h / h_max for the class threshold
struct PatchRed {
    unsigned long long xmin, ymin, xmax, ymax, hmax, hcmin;
    uint32_t hist[kHBins];
};

struct WorkItem {
    int64_t begin, end;
    int32_t patch, pad;
};

// Device views handed to the kernels.
struct State {
    double *x, *y, *z, *vx, *vy, *vz, *m, *h, *u, *du_prev, *axp, *ayp, *azp;
};

// Cell record, 16 bytes: particles [x, y) of the sorted order (x = y: empty;
// fine cells hold small particles, coarse cells big ones), z = the largest h
// in the cell (FP32 bits), w = for fine cells the tight box of the cell's
// particles, as insets from the cell faces in 1/kBoxQ of the cell edge:
// bits 0-4 low x, 5-9 high x, 10-14 low y, 15-19 high y, 20-24 low z,
// 25-29 high z (a particle with offset o lies in [lo, kBoxQ - hi) / kBoxQ of
// the edge, up to the FP32 rounding of o).
constexpr int kBoxQ = 32;
struct Grid {
    uint4* cell;         // [cell] record above
    uint32_t* cellxyz;   // [particle] cx | cy << 8 | cz << 16
    const uint16_t* patch_of;  // [particle] patch index
    float* hnb;          // [fine cell] the largest h of the fine cells within
                         // K cells along each axis (z periodic): no small
                         // particle searching from this cell meets a larger one
};

struct Recs {             // FP32 records (written by gather / density)
    float4* r4;          // {ox, oy, oz, 4 h^2}  neighbour pre-filter
    float4* r5;          // {ox, oy, oz, m}      pair sums (mixed)
    float4* rv;          // {vhx, vhy, vhz, 1/(2h)} time-centred velocity (mixed)
    float4* rt;          // {rho, P/rho^2, c, h} thermodynamics (mixed)
    float* hc;           // h/c (mixed)
    float* pf;           // P (mixed)
    float* uf;           // u, staged by the gather (mixed)
    float4* acc;         // {ax, ay, az, du} (mixed)
};

struct Fp64 {             // FP64-path fields
    double *vhx, *vhy, *vhz;   // time-centred velocity
    double *rho, *P, *c, *A, *hc;
    double *w, *w5;            // w = 1/(2h) and w^5 of the kernel gradient
    double *ax, *ay, *az, *du;
};

// ---- small device helpers ------------------------------------------------
__device__ __forceinline__ unsigned long long ord_f64(double d)
{
    unsigned long long b = (unsigned long long)__double_as_longlong(d);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__host__ __device__ __forceinline__ double unord_f64(unsigned long long u)
{
    unsigned long long b = (u >> 63) ? (u & 0x7fffffffffffffffull) : ~u;
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)b);
#else
    double d;
    memcpy(&d, &b, sizeof(d));
    return d;
#endif
}
__host__ __device__ __forceinline__ uint32_t part1by2(uint32_t v)
{
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}
__host__ __device__ __forceinline__ uint32_t compact1by2(uint32_t v)
{
    v &= 0x09249249u;
    v = (v | (v >> 2)) & 0x030C30C3u;
    v = (v | (v >> 4)) & 0x0300F00Fu;
    v = (v | (v >> 8)) & 0x030000FFu;
    v = (v | (v >> 16)) & 0x000003FFu;
    return v;
}

// ---- launch wrappers (each returns the number of kernels launched) --------
struct Launch {
    cudaStream_t stream;
    int sms;
};

int launch_reduce_bbox(const Launch& L, const State& s, const WorkItem* items, int nitems,
                       PatchRed* red);
int launch_h_hist(const Launch& L, const State& s, const WorkItem* items, int nitems, PatchRed* red);
int launch_grid_params(const Launch& L, int npatch, const PatchRed* red, PatchDev* pd,
                       double cell_factor, int* status);
int launch_keys(const Launch& L, int64_t n, const State& s, const uint16_t* patch_of,
                PatchDev* pd, uint32_t* keys, uint32_t* vals);
// LSD radix sort of (keys, vals); result in (keys, vals); uses alternates.
int launch_radix_sort(const Launch& L, int64_t n, int passes, uint32_t* keys, uint32_t* vals,
                      uint32_t* keys_alt, uint32_t* vals_alt, uint32_t* hist, uint32_t* scan_tmp);
size_t radix_hist_words(int64_t n);
// Row-length hints for the list pool: the previous lists' row lengths,
// carried into the new sorted order by the gather.  Only a hint: the list
// kernel reserves from it and repairs rows that outgrow their reservation.
constexpr uint32_t kNoHint = 0xffffffffu;
struct RowHint {
    const uint32_t* cnt_prev;    // row lengths in the previous sorted order
    const int* valid;            // nonzero: cnt_prev belongs to the order being gathered from
    uint32_t* rowcap;            // out: hint per new sorted slot, kNoHint if none
};
// hsearch (optional, the order gathered from): the h of the search when it
// is not the particles' h (the candidate superset of reused lists), gathered
// into hsearch_out and used for the search records and cell maxima
int launch_gather(const Launch& L, int64_t n, const uint32_t* skeys, const uint32_t* svals,
                  const State& src, const State& dst, const uint32_t* perm_src,
                  uint32_t* perm_dst, const PatchDev* pd, const Grid& g, const Recs& r,
                  const Fp64& f, int mixed, const RowHint& hint, const double* hsearch = nullptr,
                  double* hsearch_out = nullptr);
// the FP32 records of the current state in the current sorted order, on the
// grid of the last sort (what the gather writes, with the unscaled h)
int launch_refresh_records(const Launch& L, int64_t n, const State& s, const uint16_t* patch_of,
                           const PatchDev* pd, const uint32_t* cellxyz, const Recs& r, const Fp64& f, int mixed);
// tight boxes of the fine cells (after the gather)
int launch_cell_boxes(const Launch& L, int npatch, const PatchDev* pd, const Grid& g, const float4* r4);
// g.hnb for stencil half-extent K (tmp: one float per cell)
int launch_cell_hnb(const Launch& L, int npatch, const PatchDev* pd, const Grid& g, int K, float* tmp);
// the state's vote for the grid of the next sort (vote[0]: non-empty fine
// cells, vote[1]: those whose hnb is below 0.8 h_s in a patch with h_s above
// 1.4 h_median); vote is cleared here
int launch_cell_vote(const Launch& L, int npatch, const PatchDev* pd, const Grid& g, unsigned long long* vote);
// temporary words of the device-wide exclusive scan over n values
int64_t scan_tmp_words(int64_t n);

struct NbArgs {
    int64_t n;
    const PatchDev* pd;
    Grid g;
    const float4* r4;
    const double *x, *y, *z, *h;
    const WorkItem* units;               // 32 consecutive particles of one patch each
    int64_t nunits;
    uint32_t* cnt;                       // |N(i)|
    uint32_t* nown;                      // n_i
    unsigned long long* rowstart;        // first pool entry of row i
    uint32_t* col;                       // the list pool
    const uint32_t* rowcap;              // row-length hints (kNoHint: none)
    unsigned long long* pool_used;       // [0] entries reserved, [1] entries listed (nnz)
    int64_t max_pairs;                   // bound on nnz
    int64_t pool_cap;                    // entries the pool holds (max_pairs + slack)
    int* status;
};
// K: stencil half-extent of every patch (1 for cell_factor >= 1, 2 for >= 1/2, else 3)
// exact = 1: the neighbour lists and n_i; exact = 0: the candidate superset
// of reused lists (every candidate within the grid's scaled search radius)
int launch_nb_lists(const Launch& L, const NbArgs& a, int K, int exact);
// exact lists (a.col, a.cnt, a.nown; rows at a.rowstart) from the superset
// rows col_s / cnt_s at the same offsets, on the current records and state
int launch_nb_filter(const Launch& L, const NbArgs& a, const uint32_t* col_s, const uint32_t* cnt_s);
int launch_canonical_rows(const Launch& L, int64_t n, const unsigned long long* rowstart,
                          const uint32_t* cnt, const uint64_t* off, const uint32_t* col, uint32_t* out);
// exclusive scan of n u32 values into u64 out[0..n], out[n] = total
int launch_scan_u32_to_u64(const Launch& L, int64_t n, const uint32_t* in, uint64_t* out, uint64_t* tmp);

struct PairArgs {
    int64_t n;
    const PatchDev* pd;
    const uint16_t* patch_of;
    const unsigned long long* rowstart;  // row i is col[rowstart[i] .. + cnt[i])
    const uint32_t* cnt;
    const uint32_t* col;
    const uint32_t* cellxyz;             // [particle] cell, for kFarCode columns
    State s;
    Recs r;
    Fp64 f;
    double gamma, alpha, beta, eps;
    int kernel, kernel_n;                // SPH_KERNEL_*; n of the Sinc kernel
    int grad_h;                          // 1: grad-h form (density stores A/Omega)
    double kb;                           // sigma_W (Wendland) or B_n (Sinc)
    int* status;
    // row-length bins (nullptr order: every particle, in sorted order): the
    // launch takes positions bounds[bin_lo] .. bounds[bin_hi + 1] of order,
    // the particles whose rows fall in those octaves
    const uint32_t* order;
    const uint32_t* bounds;
    int bin_lo, bin_hi;
};
int launch_density(const Launch& L, const PairArgs& a, int tpp, int mixed);
int launch_momentum(const Launch& L, const PairArgs& a, int tpp, int mixed);
// Row-length bins: octave 0 holds the empty rows, octave o >= 1 the rows with
// |N(i)| in (2^(o-2), 2^(o-1)], o < kPairOctaves (the last octave takes every
// longer row).  With a target of 2^w list words per lane, octave o gets
// clamp(2^(o-1-w), 1, 32) lanes per particle -- the smallest power of two
// that keeps a lane at 2^w words or fewer -- and the rows of one launch's
// warps differ by less than 2x.
constexpr int kPairOctaves = 16;
__host__ __device__ __forceinline__ int octave_tpp(int o, int w)
{
    const int e = o - 1 - w;
    return e <= 0 ? 1 : (e >= 5 ? 32 : 1 << e);
}
// order = the particles stably sorted by octave (sorted order kept inside
// each octave), bounds[o] = first position of octave o, bounds[kPairOctaves] = n
int launch_pair_bins(const Launch& L, int64_t n, const uint32_t* cnt, uint32_t* keys, uint32_t* order,
                     uint32_t* keys_alt, uint32_t* vals_alt, uint32_t* hist, uint32_t* scan_tmp, uint32_t* bounds);
// the sums over row-length bins with 2^w words per lane (one launch per
// distinct lanes-per-particle value)
int launch_density_binned(const Launch& L, PairArgs a, int w, int mixed);
int launch_momentum_binned(const Launch& L, PairArgs a, int w, int mixed);
// list-free pair sums over the search of the current grid (stencil
// half-extent K); the density pass also writes |N(i)| and n_i and adds the
// pairs to pool_used[1]
int launch_fused_density(const Launch& L, const NbArgs& a, const PairArgs& pa, int K, int mixed);
int launch_fused_momentum(const Launch& L, const NbArgs& a, const PairArgs& pa, int K, int mixed);

struct StepArgs {
    int64_t n;
    PatchDev* pd;
    int npatch;
    const WorkItem* items;
    int nitems;
    PatchRed* red;
    State s;
    Recs r;
    Fp64 f;
    const uint32_t* nown;
    double courant, dt_growth, dt_fixed, n_target;
    int adapt_h, mixed;
    const double* hfac;  // [n] 0.5 (1 + cbrt(n_target / n)) for 0 < n < kHFacN, host-computed

    double* partials;    // [nitems][7]
    double* cons;        // [npatch][7]
    int* status;
};
int launch_hc_min(const Launch& L, const StepArgs& a);
int launch_dt(const Launch& L, const StepArgs& a);
int launch_update(const Launch& L, const StepArgs& a);
// reused candidate supersets: the state the superset was built on (sorted
// order), and the check that it still holds every neighbour pair
struct SkinRef {
    double *x0, *y0, *z0;  // positions the superset was built on
    double* h0;            // its search h (the superset lists r < 2 max(h0_i, h0_j))
};
int launch_skin_snapshot(const Launch& L, int64_t n, const State& s, const SkinRef& ref);
// the superset's search h per particle (current order): h (1 + skin + 3 (f - 1)+),
// f the h-adaptation factor of the last step (from n_i; 1 when nown is NULL)
int launch_skin_radius(const Launch& L, int64_t n, const State& s, const uint32_t* nown, const double* hfac,
                       double n_target, double skin, double* hsearch);
// flag (device) = 1 while max |x - x0| <= min (h0 - h), h0 = the superset's search h
int launch_skin_check(const Launch& L, int64_t n, const State& s, const uint16_t* patch_of, const PatchDev* pd,
                      const SkinRef& ref, unsigned long long* red, int* flag);
int launch_conserved_items(const Launch& L, const StepArgs& a);
int launch_conserved_finalize(const Launch& L, const StepArgs& a);
int launch_step_finalize(const Launch& L, const StepArgs& a);
int launch_unpermute_f64(const Launch& L, int64_t n, const double* src, const uint32_t* perm,
                         double* dst);
int launch_unpermute_f32(const Launch& L, int64_t n, const float* src, int stride,
                         const uint32_t* perm, double* dst);
int launch_unpermute_u32(const Launch& L, int64_t n, const uint32_t* src, const uint32_t* perm,
                         double* dst);
int launch_validate(const Launch& L, int64_t n, const State& s, int* status);
int launch_reset_red(const Launch& L, int npatch, PatchRed* red);

}  // namespace sphg
