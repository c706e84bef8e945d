// sph_api.cu -- the C ABI declared in include/sph.h: context, device memory,
// the order of the phases of one timestep, CUDA-graph replay, phase timers,
// checkpoints and the launch autotuner.  All device work is issued on the
// context's stream; the kernels live in sph_sort.cu, sph_neighbors.cu,
// sph_pairs.cu and sph_step.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "sph_internal.cuh"

using namespace sphg;

namespace {

thread_local std::string g_last_error = "";

bool is_sticky(cudaError_t e)
{
    switch (e) {
    case cudaErrorIllegalAddress:
    case cudaErrorLaunchFailure:
    case cudaErrorIllegalInstruction:
    case cudaErrorMisalignedAddress:
    case cudaErrorInvalidAddressSpace:
    case cudaErrorInvalidPc:
    case cudaErrorHardwareStackError:
    case cudaErrorAssert:
    case cudaErrorLaunchTimeout:
    case cudaErrorECCUncorrectable:
        return true;
    default:
        return false;
    }
}

__global__ void k_iota(int64_t n, uint32_t* p)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = (uint32_t)i;
}

// dst[perm[k]] = src[k]: a sorted-order array back to the caller's order
__global__ void k_scatter_u32(int64_t n, const uint32_t* src, const uint32_t* perm, uint32_t* dst)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        dst[perm[k]] = src[k];
}

// dst[k] = src[perm[k]]: a caller's-order array into a sorted order; a
// permutation entry out of range (a damaged state buffer) gives 0
__global__ void k_gather_u32(int64_t n, const uint32_t* src, const uint32_t* perm, uint32_t* dst)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t j = perm[k];
        dst[k] = (int64_t)j < n ? src[j] : 0u;
    }
}

__global__ void k_accum_pairs(const unsigned long long* total, unsigned long long* acc, const int* status)
{
    if (!(*status & kStBad)) *acc += *total;
}

__global__ void k_fill_patch_of(const WorkItem* items, int nitems, uint16_t* patch_of)
{
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const WorkItem w = items[it];
        for (int64_t i = w.begin + threadIdx.x; i < w.end; i += blockDim.x) patch_of[i] = (uint16_t)w.patch;
    }
}

}  // namespace

struct sph_ctx {
    sph_config cfg;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int sms = 1;
    std::string err;
    bool poisoned = false;

    int64_t cap_n = 0, max_pairs = 0, pool_cap = 0, cap_cells = 0;
    int64_t cells_used = 0;        // cell-table records the patches' slices span
    int cap_patch = 0, cap_items = 0;
    int64_t n = 0;
    int npatch = 0, nitems = 0, radix_passes = 3;
    int tpp_pair = 8;              // lanes per particle of the momentum sum
    int tpp_den = 8;               // ... and of the density sum
    // row-length bins of the pair sums: log2 of the list words per lane
    // (0: every particle with the uniform tpp above)
    int bins_pair = 0, bins_den = 0;
    uint32_t* bin_order = nullptr; // particles sorted stably by row-length octave
    uint32_t* bin_bounds = nullptr; // [kPairOctaves + 1] octave starts in bin_order
    bool bins_valid = false;       // bin_order belongs to the current lists
    double cell_factor = 0.5;
    // the cell factor came from the default or the autotuner: between 1/2 and
    // 0.4 it follows the cell grid's vote (cf_vote, taken at every sort)
    bool cf_auto = true;
    unsigned long long* cf_vote = nullptr;
    unsigned long long* h_cf_vote = nullptr;   // pinned
    int64_t cf_switches = 0;
    int mixed = 1;
    bool fused = false;            // pair sums without lists (SPH_PAIRS_FUSED in effect)
    // reused candidate supersets (list_skin > 0, list mode)
    double skin = 0.0;
    bool sup_valid = false;        // the superset of the current order still holds every pair
    uint32_t *col_s = nullptr, *cnt_s = nullptr;  // superset pool and row lengths (rows at rowstart)
    int* hint_ok_s = nullptr;      // device flag: cnt_s holds row lengths of the current order
    int64_t max_pairs_s = 0;
    SkinRef skinref{};
    double* hsearch_pre = nullptr; // search h of a superset build, order before its sort
    unsigned long long* skin_red = nullptr;
    int* skin_flag = nullptr;
    int* h_skin_flag = nullptr;    // pinned
    int64_t rebuilds = 0;          // superset builds so far

    State st[2];
    int cur = 0;
    uint32_t* perm[2] = {nullptr, nullptr};
    uint16_t* patch_of = nullptr;
    uint32_t *keys = nullptr, *vals = nullptr, *keys_alt = nullptr, *vals_alt = nullptr;
    float* hnb_tmp = nullptr;   // one float per cell: the x-y pass of the grid's hnb
    uint32_t *hist = nullptr, *scan32 = nullptr;
    Grid grid{};
    Recs rec{};
    Fp64 f64{};
    uint32_t *cnt = nullptr, *nown = nullptr, *col = nullptr, *col_plain = nullptr;
    WorkItem* units = nullptr;     // 32-particle warp units, per patch
    int64_t nunits = 0, cap_units = 0;
    unsigned long long *rowstart = nullptr, *pool_used = nullptr;  // pool_used: [reserved, listed]
    uint32_t* rowcap = nullptr;    // row-length hints in the current sorted order
    int* hint_ok = nullptr;        // device flag: cnt holds row lengths of the current order
    bool cnt_valid = false;        // host: cnt holds the row lengths of the current order
    uint32_t* cnt_orig = nullptr;  // row lengths carried to the caller's order (set_particles)
    uint64_t* scan64 = nullptr;
    bool canon_valid = false;      // off / col_plain hold the canonical CSR
    int64_t col_plain_cap = 0;
    uint64_t* off = nullptr;
    PatchDev* pd = nullptr;
    PatchRed* red = nullptr;
    WorkItem* items = nullptr;
    double *partials = nullptr, *cons = nullptr, *scratch = nullptr;
    double* hfac = nullptr;        // h-adaptation factors by neighbour count
    double kernel_b = 0.0;         // sigma_W (Wendland) or B_n (Sinc)
    int* status = nullptr;
    int* h_status = nullptr;     // pinned
    unsigned long long* pair_acc = nullptr;  // sum of |N| over the steps taken
    std::vector<int64_t> patch_off;

    bool nb_valid = false, rho_valid = false, acc_valid = false;
    bool fresh = true;           // no sort since set_particles / set_state
    int64_t nnz = -1;

    bool prof = false;
    double prof_ms[SPH_PHASE_COUNT] = {};
    int64_t prof_launch[SPH_PHASE_COUNT] = {};
    std::vector<cudaEvent_t> ev_free;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> marks;
    int64_t launches = 0;

    // captured steps by buffer parity and kind (1: with the sort and search,
    // 0: on a reused superset)
    cudaGraphExec_t gexec[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    int64_t graph_kernels[2][2] = {{0, 0}, {0, 0}};

    std::vector<void*> allocs;
};

namespace {

sph_status fail(sph_ctx* c, sph_status s, const std::string& msg)
{
    if (c) c->err = msg;
    g_last_error = msg;
    return s;
}

sph_status cuda_fail(sph_ctx* c, cudaError_t e, const char* where)
{
    std::string msg = std::string(where) + ": " + cudaGetErrorString(e);
    if (is_sticky(e)) {
        if (c) c->poisoned = true;
        return fail(c, SPH_ESTATE, msg + " (context poisoned)");
    }
    return fail(c, SPH_ECUDA, msg);
}

#define CK(call)                                                   \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);   \
    } while (0)

template <typename T>
bool dalloc(sph_ctx* ctx, T*& p, size_t count)
{
    void* q = nullptr;
    size_t bytes = count * sizeof(T);
    if (bytes == 0) bytes = 16;
    if (cudaMalloc(&q, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
        return false;
    }
    ctx->allocs.push_back(q);
    p = (T*)q;
    return true;
}

Launch launch_of(const sph_ctx* ctx) { return Launch{ctx->stream, ctx->sms}; }

void destroy_graphs(sph_ctx* ctx)
{
    for (int k = 0; k < 2; k++)
        for (int r = 0; r < 2; r++) {
            if (ctx->gexec[k][r]) cudaGraphExecDestroy(ctx->gexec[k][r]);
            ctx->gexec[k][r] = nullptr;
            ctx->graph_kernels[k][r] = 0;
        }
}

// ---- phase timers -----------------------------------------------------------
cudaEvent_t get_event(sph_ctx* ctx)
{
    if (!ctx->ev_free.empty()) {
        cudaEvent_t e = ctx->ev_free.back();
        ctx->ev_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

struct Phase {
    sph_ctx* ctx;
    int ph;
    cudaEvent_t a = nullptr;
    int64_t l0;
    Phase(sph_ctx* c, int p) : ctx(c), ph(p), l0(c->launches)
    {
        if (ctx->prof) {
            a = get_event(ctx);
            cudaEventRecord(a, ctx->stream);
        }
    }
    ~Phase()
    {
        if (ctx->prof) {
            cudaEvent_t b = get_event(ctx);
            cudaEventRecord(b, ctx->stream);
            ctx->marks.push_back({ph, {a, b}});
            ctx->prof_launch[ph] += ctx->launches - l0;
        }
    }
};

void collect_profile(sph_ctx* ctx)
{
    if (ctx->marks.empty()) return;
    cudaStreamSynchronize(ctx->stream);
    for (auto& m : ctx->marks) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, m.second.first, m.second.second) == cudaSuccess)
            ctx->prof_ms[m.first] += ms;
        ctx->ev_free.push_back(m.second.first);
        ctx->ev_free.push_back(m.second.second);
    }
    ctx->marks.clear();
}

// ---- kernel normalisation -------------------------------------------------------
// Wendland (Eq. 2): sigma_W = 21 / (16 pi).  Sinc (Sec. 3): B_n from
// 4 pi B_n int_0^2 v^2 sinc^n(pi v / 2) dv = 1, the integral by composite
// 5-point Gauss-Legendre quadrature on 400 panels (the integrand is smooth).
double kernel_norm(int kernel, int n)
{
    const double pi = 3.14159265358979323846;
    if (kernel != SPH_KERNEL_SINC) return 21.0 / (16.0 * pi);
    const double xg[5] = {0.0, -0.5384693101056831, 0.5384693101056831, -0.9061798459386640, 0.9061798459386640};
    const double wg[5] = {0.5688888888888889, 0.4786286704993665, 0.4786286704993665, 0.2369268850561891,
                          0.2369268850561891};
    const int panels = 400;
    const double hw = 1.0 / panels;  // half width of a panel on [0, 2]
    double total = 0.0;
    for (int p = 0; p < panels; p++) {
        const double mid = (2.0 * p + 1.0) * hw;
        for (int k = 0; k < 5; k++) {
            const double v = mid + hw * xg[k];
            const double x = 0.5 * pi * v;
            const double s = x == 0.0 ? 1.0 : std::sin(x) / x;
            double sn = 1.0;
            for (int e = 0; e < n; e++) sn *= s;
            total += wg[k] * hw * v * v * sn;
        }
    }
    return 1.0 / (4.0 * pi * total);
}

// ---- argument bundles ---------------------------------------------------------
NbArgs nb_args(sph_ctx* ctx)
{
    NbArgs a;
    a.n = ctx->n;
    a.pd = ctx->pd;
    a.g = ctx->grid;
    a.r4 = ctx->rec.r4;
    const State& s = ctx->st[ctx->cur];
    a.x = s.x; a.y = s.y; a.z = s.z; a.h = s.h;
    a.cnt = ctx->cnt;
    a.nown = ctx->nown;
    a.rowstart = ctx->rowstart;
    a.col = ctx->col;
    a.rowcap = ctx->rowcap;
    a.pool_used = ctx->pool_used;
    a.max_pairs = ctx->max_pairs;
    a.pool_cap = ctx->pool_cap;
    a.status = ctx->status;
    a.units = ctx->units;
    a.nunits = ctx->nunits;
    return a;
}

PairArgs pair_args(sph_ctx* ctx)
{
    PairArgs a;
    a.n = ctx->n;
    a.pd = ctx->pd;
    a.patch_of = ctx->patch_of;
    a.rowstart = ctx->rowstart;
    a.cnt = ctx->cnt;
    a.col = ctx->col;
    a.cellxyz = ctx->grid.cellxyz;
    a.s = ctx->st[ctx->cur];
    a.r = ctx->rec;
    a.f = ctx->f64;
    a.gamma = ctx->cfg.gamma;
    a.alpha = ctx->cfg.av_alpha;
    a.beta = ctx->cfg.av_beta;
    a.eps = ctx->cfg.av_eps;
    a.kernel = ctx->cfg.kernel;
    a.kernel_n = ctx->cfg.kernel_n;
    a.grad_h = ctx->cfg.grad_h;
    a.kb = ctx->kernel_b;
    a.status = ctx->status;
    a.order = nullptr;
    a.bounds = nullptr;
    a.bin_lo = a.bin_hi = 0;
    return a;
}

StepArgs step_args(sph_ctx* ctx)
{
    StepArgs a;
    a.n = ctx->n;
    a.pd = ctx->pd;
    a.npatch = ctx->npatch;
    a.items = ctx->items;
    a.nitems = ctx->nitems;
    a.red = ctx->red;
    a.s = ctx->st[ctx->cur];
    a.r = ctx->rec;
    a.f = ctx->f64;
    a.nown = ctx->nown;
    a.courant = ctx->cfg.courant;
    a.dt_growth = ctx->cfg.dt_growth;
    a.dt_fixed = ctx->cfg.dt_fixed;
    a.n_target = ctx->cfg.n_target;
    a.adapt_h = ctx->cfg.adapt_h;
    a.mixed = ctx->mixed;
    a.hfac = ctx->hfac;
    a.partials = ctx->partials;
    a.cons = ctx->cons;
    a.status = ctx->status;
    return a;
}

// ---- the phases (asynchronous, no host synchronisation) -----------------------
// superset: the sort and cells of a candidate superset (reused lists): the
// search h of every particle grown by its skin, gathered into skinref.h0;
// the row-length hints come from the superset's rows
void enqueue_sort(sph_ctx* ctx, bool superset = false)
{
    const Launch L = launch_of(ctx);
    State s = ctx->st[ctx->cur];
    if (superset) {
        const bool have_n = !ctx->fresh && ctx->cfg.adapt_h;
        ctx->launches += launch_skin_radius(L, ctx->n, ctx->st[ctx->cur], have_n ? ctx->nown : nullptr, ctx->hfac,
                                            ctx->cfg.n_target, ctx->skin, ctx->hsearch_pre);
        s.h = ctx->hsearch_pre;
    }
    {
        Phase p(ctx, SPH_PHASE_BBOX);
        ctx->launches += launch_reset_red(L, ctx->npatch, ctx->red);
        ctx->launches += launch_reduce_bbox(L, s, ctx->items, ctx->nitems, ctx->red);
        ctx->launches += launch_h_hist(L, s, ctx->items, ctx->nitems, ctx->red);
        ctx->launches += launch_grid_params(L, ctx->npatch, ctx->red, ctx->pd, ctx->cell_factor, ctx->status);
    }
    {
        Phase p(ctx, SPH_PHASE_KEYS);
        ctx->launches += launch_keys(L, ctx->n, s, ctx->patch_of, ctx->pd, ctx->keys, ctx->vals);
    }
    {
        Phase p(ctx, SPH_PHASE_SORT);
        ctx->launches += launch_radix_sort(L, ctx->n, ctx->radix_passes, ctx->keys, ctx->vals, ctx->keys_alt,
                                           ctx->vals_alt, ctx->hist, ctx->scan32);
    }
    {
        Phase p(ctx, SPH_PHASE_GATHER);
        cudaMemsetAsync(ctx->grid.cell, 0, (size_t)ctx->cells_used * sizeof(uint4), ctx->stream);
        const int nxt = 1 - ctx->cur;
        ctx->launches += launch_gather(L, ctx->n, ctx->keys, ctx->vals, ctx->st[ctx->cur], ctx->st[nxt],
                                       ctx->perm[ctx->cur], ctx->perm[nxt], ctx->pd, ctx->grid, ctx->rec,
                                       ctx->f64, ctx->mixed,
                                       superset ? RowHint{ctx->cnt_s, ctx->hint_ok_s, ctx->rowcap}
                                                : RowHint{ctx->cnt, ctx->hint_ok, ctx->rowcap},
                                       superset ? ctx->hsearch_pre : nullptr, superset ? ctx->skinref.h0 : nullptr);
        ctx->launches += launch_cell_boxes(L, ctx->npatch, ctx->pd, ctx->grid, ctx->rec.r4);
        ctx->launches += launch_cell_hnb(L, ctx->npatch, ctx->pd, ctx->grid, stencil_k(ctx->cell_factor), ctx->hnb_tmp);
        ctx->launches += launch_cell_vote(L, ctx->npatch, ctx->pd, ctx->grid, ctx->cf_vote);
        ctx->cur = nxt;
    }
    ctx->fresh = false;
}

void enqueue_lists(sph_ctx* ctx)
{
    const Launch L = launch_of(ctx);
    const NbArgs a = nb_args(ctx);
    {
        Phase p(ctx, SPH_PHASE_NB_RESET);
        cudaMemsetAsync(ctx->pool_used, 0, 2 * sizeof(unsigned long long), ctx->stream);
    }
    ctx->canon_valid = false;
    {
        Phase p(ctx, SPH_PHASE_NB);
        ctx->launches += launch_nb_lists(L, a, stencil_k(ctx->cell_factor), 1);
    }
    ctx->bins_valid = false;
    // the row lengths now belong to the current order: hints for the next sort
    cudaMemsetAsync(ctx->hint_ok, 1, sizeof(int), ctx->stream);
}

// the particles binned by row length, once per set of lists (counted in the
// phase that first needs them)
void enqueue_bins(sph_ctx* ctx)
{
    if (ctx->bins_valid) return;
    ctx->launches += launch_pair_bins(launch_of(ctx), ctx->n, ctx->cnt, ctx->keys, ctx->bin_order, ctx->keys_alt,
                                      ctx->vals_alt, ctx->hist, ctx->scan32, ctx->bin_bounds);
    ctx->bins_valid = true;
}

PairArgs binned_args(sph_ctx* ctx)
{
    PairArgs a = pair_args(ctx);
    a.order = ctx->bin_order;
    a.bounds = ctx->bin_bounds;
    return a;
}

void enqueue_density(sph_ctx* ctx)
{
    if (ctx->fused) {
        {
            // the density pass counts the pairs again
            Phase p(ctx, SPH_PHASE_NB_RESET);
            cudaMemsetAsync(ctx->pool_used + 1, 0, sizeof(unsigned long long), ctx->stream);
        }
        Phase p(ctx, SPH_PHASE_DENSITY);
        ctx->launches += launch_fused_density(launch_of(ctx), nb_args(ctx), pair_args(ctx),
                                              stencil_k(ctx->cell_factor), ctx->mixed);
        // cnt now holds the row lengths of the current order: hints for the next sort
        cudaMemsetAsync(ctx->hint_ok, 1, sizeof(int), ctx->stream);
        return;
    }
    Phase p(ctx, SPH_PHASE_DENSITY);
    if (ctx->bins_den) {
        enqueue_bins(ctx);
        ctx->launches += launch_density_binned(launch_of(ctx), binned_args(ctx), ctx->bins_den, ctx->mixed);
    } else {
        ctx->launches += launch_density(launch_of(ctx), pair_args(ctx), ctx->tpp_den, ctx->mixed);
    }
}

void enqueue_momentum(sph_ctx* ctx)
{
    Phase p(ctx, SPH_PHASE_MOMENTUM);
    if (ctx->fused)
        ctx->launches += launch_fused_momentum(launch_of(ctx), nb_args(ctx), pair_args(ctx),
                                               stencil_k(ctx->cell_factor), ctx->mixed);
    else if (ctx->bins_pair) {
        enqueue_bins(ctx);
        ctx->launches += launch_momentum_binned(launch_of(ctx), binned_args(ctx), ctx->bins_pair, ctx->mixed);
    } else {
        ctx->launches += launch_momentum(launch_of(ctx), pair_args(ctx), ctx->tpp_pair, ctx->mixed);
    }
}

// the candidate superset of reused lists on the grid of the last sort (its
// radius scaled by 1 + skin), and the state it was built on
void enqueue_superset(sph_ctx* ctx)
{
    const Launch L = launch_of(ctx);
    NbArgs a = nb_args(ctx);
    a.h = ctx->skinref.h0;       // the search h (no exact decisions in a superset)
    a.col = ctx->col_s;
    a.cnt = ctx->cnt_s;
    a.max_pairs = ctx->max_pairs_s;
    {
        Phase p(ctx, SPH_PHASE_NB_RESET);
        cudaMemsetAsync(ctx->pool_used, 0, 2 * sizeof(unsigned long long), ctx->stream);
    }
    {
        Phase p(ctx, SPH_PHASE_NB);
        ctx->launches += launch_nb_lists(L, a, stencil_k(ctx->cell_factor), 0);
        ctx->launches += launch_skin_snapshot(L, ctx->n, ctx->st[ctx->cur], ctx->skinref);
    }
    cudaMemsetAsync(ctx->hint_ok_s, 1, sizeof(int), ctx->stream);
}

// the exact lists of the current state from the superset: records of the
// current positions and h on the grid of the last sort, then the filter
void enqueue_filter(sph_ctx* ctx)
{
    const Launch L = launch_of(ctx);
    {
        Phase p(ctx, SPH_PHASE_GATHER);
        ctx->launches += launch_refresh_records(L, ctx->n, ctx->st[ctx->cur], ctx->patch_of, ctx->pd,
                                                ctx->grid.cellxyz, ctx->rec, ctx->f64, ctx->mixed);
    }
    {
        Phase p(ctx, SPH_PHASE_NB_RESET);
        cudaMemsetAsync(ctx->pool_used + 1, 0, sizeof(unsigned long long), ctx->stream);
    }
    ctx->canon_valid = false;
    {
        Phase p(ctx, SPH_PHASE_NB);
        ctx->launches += launch_nb_filter(L, nb_args(ctx), ctx->col_s, ctx->cnt_s);
    }
    ctx->bins_valid = false;
    cudaMemsetAsync(ctx->hint_ok, 1, sizeof(int), ctx->stream);
}

bool reuse_lists(const sph_ctx* ctx) { return ctx->skin > 0.0 && !ctx->fused; }

// density, dt, momentum, update (the step after its neighbour phase)
void enqueue_pair_phases(sph_ctx* ctx)
{
    enqueue_density(ctx);
    const Launch L = launch_of(ctx);
    {
        Phase p(ctx, SPH_PHASE_UPDATE);
        const StepArgs a = step_args(ctx);
        k_accum_pairs<<<1, 1, 0, ctx->stream>>>(ctx->pool_used + 1, ctx->pair_acc, ctx->status);
        ctx->launches += 1;
        ctx->launches += launch_hc_min(L, a);
        ctx->launches += launch_dt(L, a);
    }
    enqueue_momentum(ctx);
    {
        Phase p(ctx, SPH_PHASE_UPDATE);
        const StepArgs a = step_args(ctx);
        ctx->launches += launch_update(L, a);
        ctx->launches += launch_step_finalize(L, a);
        if (reuse_lists(ctx))
            ctx->launches += launch_skin_check(L, ctx->n, ctx->st[ctx->cur], ctx->patch_of, ctx->pd, ctx->skinref,
                                               ctx->skin_red, ctx->skin_flag);
    }
}

// one step; with reused lists, rebuild = 0 filters the current superset
// instead of sorting and searching
void enqueue_step(sph_ctx* ctx, bool rebuild = true)
{
    if (reuse_lists(ctx)) {
        if (rebuild) {
            enqueue_sort(ctx, true);
            enqueue_superset(ctx);
        }
        enqueue_filter(ctx);
    } else {
        enqueue_sort(ctx);
        if (!ctx->fused) enqueue_lists(ctx);
    }
    enqueue_pair_phases(ctx);
}

sph_status check_status(sph_ctx* ctx, const char* where)
{
    cudaError_t e = cudaMemcpyAsync(ctx->h_status, ctx->status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, where);
    collect_profile(ctx);
    const int st = *ctx->h_status;
    if (st & kStOverflow)
        return fail(ctx, SPH_EOVERFLOW, std::string(where) + ": neighbour lists exceed max_pairs");
    if (st & kStNonFinite) return fail(ctx, SPH_ENONFINITE, std::string(where) + ": non-finite value");
    if (st & kStTimeout) return fail(ctx, SPH_ETIMEOUT, std::string(where) + ": device wait timed out");
    return SPH_OK;
}

sph_status begin_call(sph_ctx* ctx)
{
    if (!ctx) return fail(nullptr, SPH_EINVAL, "null context");
    if (ctx->poisoned) return fail(ctx, SPH_ESTATE, "context poisoned by an earlier CUDA error");
    cudaError_t e = cudaMemsetAsync(ctx->status, 0, sizeof(int), ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "status reset");
    return SPH_OK;
}

sph_status after_launches(sph_ctx* ctx, const char* where)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, where);
    return SPH_OK;
}

// patch table for the given original-order offsets (slots == original order)
sph_status setup_patches(sph_ctx* ctx, int np, const int64_t* offsets)
{
    std::vector<PatchDev> pd(np);
    std::vector<WorkItem> items;
    int64_t cbase = 0;
    for (int p = 0; p < np; p++) {
        PatchDev P;
        memset(&P, 0, sizeof(P));
        P.begin = offsets[p];
        P.end = offsets[p + 1];
        const int64_t np_ = P.end - P.begin;
        int64_t cap = 2 * np_ + 4096;
        const int64_t maxc = (int64_t)kMaxCellsAxis * kMaxCellsAxis * kMaxCellsAxis * 9 / 8 + 64;
        if (cap > maxc) cap = maxc;
        P.cell_base = cbase;
        P.cell_cap = cap;
        cbase += cap;
        P.lz = ctx->cfg.lz;
        P.item_begin = (int)items.size();
        for (int64_t b = P.begin; b < P.end; b += kItemChunk) {
            WorkItem w;
            w.begin = b;
            w.end = b + kItemChunk < P.end ? b + kItemChunk : P.end;
            w.patch = p;
            w.pad = 0;
            items.push_back(w);
        }
        P.item_end = (int)items.size();
        pd[p] = P;
    }
    // the same patch layout as the current one (a state or particle set
    // uploaded again): the work tables on the device still hold it
    const bool same = ctx->npatch == np && (int64_t)ctx->patch_off.size() == (int64_t)np + 1 &&
                      std::equal(offsets, offsets + np + 1, ctx->patch_off.begin()) &&
                      ctx->nitems == (int)items.size();
    std::vector<WorkItem> units;
    for (int p = 0; p < np && !same; p++) {
        for (int64_t b = offsets[p]; b < offsets[p + 1]; b += 32) {
            WorkItem w;
            w.begin = b;
            w.end = b + 32 < offsets[p + 1] ? b + 32 : offsets[p + 1];
            w.patch = p;
            w.pad = 0;
            units.push_back(w);
        }
    }
    if (cbase > ctx->cap_cells || (int)items.size() > ctx->cap_items || (int64_t)units.size() > ctx->cap_units)
        return fail(ctx, SPH_EINVAL, "patch table exceeds capacity");
    if (!same) {
        if (!units.empty())
            CK(cudaMemcpyAsync(ctx->units, units.data(), sizeof(WorkItem) * units.size(), cudaMemcpyHostToDevice,
                               ctx->stream));
        ctx->nunits = (int64_t)units.size();
    }
    CK(cudaMemcpyAsync(ctx->pd, pd.data(), sizeof(PatchDev) * np, cudaMemcpyHostToDevice, ctx->stream));
    if (!items.empty() && !same)
        CK(cudaMemcpyAsync(ctx->items, items.data(), sizeof(WorkItem) * items.size(), cudaMemcpyHostToDevice,
                           ctx->stream));
    ctx->npatch = np;
    ctx->nitems = (int)items.size();
    ctx->cells_used = cbase;
    if (ctx->nitems > 0 && !same) {
        const int grid = ctx->nitems < ctx->sms * 8 ? ctx->nitems : ctx->sms * 8;
        k_fill_patch_of<<<grid, 256, 0, ctx->stream>>>(ctx->items, ctx->nitems, ctx->patch_of);
    }
    int bits = 0;
    while ((1 << bits) < np) bits++;
    ctx->radix_passes = (kPatchShift + bits + 7) / 8;
    ctx->patch_off.assign(offsets, offsets + np + 1);
    ctx->nb_valid = ctx->rho_valid = ctx->acc_valid = ctx->sup_valid = false;
    ctx->cnt_valid = false;
    destroy_graphs(ctx);
    // new particle order: no row-length hints
    CK(cudaMemsetAsync(ctx->hint_ok, 0, sizeof(int), ctx->stream));
    if (ctx->hint_ok_s) CK(cudaMemsetAsync(ctx->hint_ok_s, 0, sizeof(int), ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return after_launches(ctx, "setup_patches");
}

double* state_field(State& s, int k)
{
    double* f[13] = {s.x, s.y, s.z, s.vx, s.vy, s.vz, s.m, s.h, s.u, s.du_prev, s.axp, s.ayp, s.azp};
    return f[k];
}

}  // namespace

// ============================================================================
extern "C" {

void sph_config_default(sph_config* c)
{
    if (!c) return;
    memset(c, 0, sizeof(*c));
    c->precision = SPH_MIXED;
    c->kernel = SPH_KERNEL_WENDLAND;
    c->kernel_n = 6;
    c->gamma = 5.0 / 3.0;
    c->n_target = 100.0;
    c->courant = 0.2;
    c->dt_growth = 1.1;
    c->av_alpha = 1.0;
    c->av_beta = 2.0;
    c->av_eps = 0.01;
    c->lz = 1.0;
    c->dt_fixed = 0.0;
    c->adapt_h = 1;
    c->threads_per_particle = 0;
    c->cell_factor = 0.0;       // automatic: 1/2, then as the cell grid votes
    c->max_particles = 1 << 20;
    c->max_pairs = 0;
    c->max_patches = 1;
    c->use_graph = 0;
    c->pair_bins = 0;
    c->reserved = 0;
    c->cuda_stream = nullptr;
}

const char* sph_status_string(sph_status s)
{
    switch (s) {
    case SPH_OK: return "SPH_OK";
    case SPH_EINVAL: return "SPH_EINVAL";
    case SPH_ENOMEM: return "SPH_ENOMEM";
    case SPH_ECUDA: return "SPH_ECUDA";
    case SPH_EOVERFLOW: return "SPH_EOVERFLOW";
    case SPH_ENONFINITE: return "SPH_ENONFINITE";
    case SPH_ETIMEOUT: return "SPH_ETIMEOUT";
    case SPH_ESTATE: return "SPH_ESTATE";
    }
    return "unknown";
}

const char* sph_last_error(const sph_ctx* ctx)
{
    if (ctx) return ctx->err.c_str();
    return g_last_error.c_str();
}

void sph_destroy(sph_ctx* ctx)
{
    if (!ctx) return;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    destroy_graphs(ctx);
    for (auto& m : ctx->marks) {
        cudaEventDestroy(m.second.first);
        cudaEventDestroy(m.second.second);
    }
    for (auto e : ctx->ev_free) cudaEventDestroy(e);
    for (void* p : ctx->allocs)
        if (p) cudaFree(p);
    if (ctx->h_status) cudaFreeHost(ctx->h_status);
    if (ctx->h_skin_flag) cudaFreeHost(ctx->h_skin_flag);
    if (ctx->h_cf_vote) cudaFreeHost(ctx->h_cf_vote);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

sph_status sph_create(const sph_config* cfg_in, sph_ctx** out)
{
    if (!out) return fail(nullptr, SPH_EINVAL, "out is NULL");
    *out = nullptr;
    sph_config cfg;
    if (cfg_in) cfg = *cfg_in;
    else sph_config_default(&cfg);
    if (cfg.precision != SPH_FP64 && cfg.precision != SPH_MIXED)
        return fail(nullptr, SPH_EINVAL, "precision must be SPH_FP64 or SPH_MIXED");
    if (cfg.kernel != SPH_KERNEL_WENDLAND && cfg.kernel != SPH_KERNEL_SINC)
        return fail(nullptr, SPH_EINVAL, "unsupported kernel");
    if (cfg.kernel == SPH_KERNEL_SINC && !(cfg.kernel_n >= 2 && cfg.kernel_n <= 16))
        return fail(nullptr, SPH_EINVAL, "kernel_n must be in [2, 16] for the Sinc kernel");
    if (cfg.grad_h != 0 && cfg.grad_h != 1) return fail(nullptr, SPH_EINVAL, "grad_h must be 0 or 1");
    if (!(cfg.list_skin >= 0.0 && cfg.list_skin <= 1.0))
        return fail(nullptr, SPH_EINVAL, "list_skin must be in [0, 1]");
    if (cfg.pair_mode != SPH_PAIRS_LISTS && cfg.pair_mode != SPH_PAIRS_FUSED && cfg.pair_mode != SPH_PAIRS_AUTO)
        return fail(nullptr, SPH_EINVAL, "pair_mode must be SPH_PAIRS_LISTS, SPH_PAIRS_FUSED or SPH_PAIRS_AUTO");
    if (cfg.max_particles < 1 || cfg.max_particles > kMaxParticles)
        return fail(nullptr, SPH_EINVAL, "max_particles must be in [1, 2^25]");
    if (cfg.max_patches < 1 || cfg.max_patches > kMaxPatches)
        return fail(nullptr, SPH_EINVAL, "max_patches must be in [1, 256]");
    const bool cf_default = cfg.cell_factor == 0.0;
    if (cfg.cell_factor == 0.0) cfg.cell_factor = 0.5;
    if (!(cfg.cell_factor >= 1.0 / 3.0 && cfg.cell_factor <= 4.0))
        return fail(nullptr, SPH_EINVAL, "cell_factor must be in [1/3, 4]");
    const int t = cfg.threads_per_particle;
    if (!(t == 0 || t == 1 || t == 2 || t == 4 || t == 8 || t == 16 || t == 32))
        return fail(nullptr, SPH_EINVAL, "threads_per_particle must be 0, 1, 2, 4, 8, 16 or 32");
    const int pb = cfg.pair_bins;
    if (!(pb == 0 || pb == -1 || pb == 8 || pb == 16 || pb == 32 || pb == 64 || pb == 128 || pb == 256))
        return fail(nullptr, SPH_EINVAL, "pair_bins must be 0, -1, 8, 16, 32, 64, 128 or 256");
    if (!(cfg.gamma > 1.0) || !(cfg.courant > 0.0) || !(cfg.dt_growth >= 1.0) || !(cfg.lz > 0.0) ||
        !(cfg.n_target > 0.0) || !(cfg.av_alpha >= 0.0) || !(cfg.av_beta >= 0.0) || !(cfg.av_eps > 0.0) ||
        !(cfg.dt_fixed >= 0.0))
        return fail(nullptr, SPH_EINVAL, "invalid physical parameter");
    if (cfg.max_pairs < 0) return fail(nullptr, SPH_EINVAL, "max_pairs < 0");

    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev < 1) {
        cudaGetLastError();
        return fail(nullptr, SPH_ECUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
    }
    sph_ctx* ctx = new (std::nothrow) sph_ctx();
    if (!ctx) return fail(nullptr, SPH_ENOMEM, "host allocation failed");
    ctx->cfg = cfg;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, dev);
    if (cfg.cuda_stream) {
        ctx->stream = (cudaStream_t)cfg.cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete ctx;
            return fail(nullptr, SPH_ECUDA, "stream creation failed");
        }
        ctx->own_stream = true;
    }
    ctx->mixed = cfg.precision == SPH_MIXED;
    ctx->kernel_b = kernel_norm(cfg.kernel, cfg.kernel_n);
    ctx->cell_factor = cfg.cell_factor;
    ctx->cf_auto = cf_default;
    if (t) ctx->tpp_pair = ctx->tpp_den = t;
    if (pb > 0) {
        int w = 0;
        while ((1 << w) < pb) w++;
        ctx->bins_pair = ctx->bins_den = w;
    }
    ctx->fused = cfg.pair_mode == SPH_PAIRS_FUSED;
    ctx->cap_n = cfg.max_particles;
    ctx->cap_patch = cfg.max_patches;
    ctx->max_pairs = cfg.max_pairs > 0 ? cfg.max_pairs : 160 * cfg.max_particles;
    // rows are reserved ahead in multiples of 8 entries, at 4/3 of their
    // previous length plus 8, and a row that outgrows its reservation takes a
    // second one: 5/2 max_pairs + 24 per particle holds any step whose lists
    // fit in max_pairs after a step whose lists did
    ctx->pool_cap = ctx->max_pairs * 5 / 2 + 24 * cfg.max_particles + 64;
    ctx->skin = cfg.list_skin;
    if (ctx->skin > 0.0) {
        // the superset lists pairs within (1 + skin) times the radius: about
        // (1 + skin)^3 as many; the exact rows sit at the superset's offsets,
        // so both pools take the superset's size
        const double g = 1.0 + ctx->skin;
        ctx->max_pairs_s = (int64_t)((double)ctx->max_pairs * g * g * g * 1.1) + 64;
        ctx->pool_cap = ctx->max_pairs_s * 5 / 2 + 24 * cfg.max_particles + 64;
    }
    ctx->cap_items = (int)(ctx->cap_n / kItemChunk + ctx->cap_patch + 1);
    ctx->cap_cells = 2 * ctx->cap_n + (int64_t)4096 * ctx->cap_patch;
    const size_t N = (size_t)ctx->cap_n;

    bool ok = true;
    for (int b = 0; b < 2 && ok; b++) {
        State& s = ctx->st[b];
        double** f[13] = {&s.x, &s.y, &s.z, &s.vx, &s.vy, &s.vz, &s.m, &s.h, &s.u, &s.du_prev, &s.axp, &s.ayp, &s.azp};
        for (int k = 0; k < 13 && ok; k++) ok = dalloc(ctx, *f[k], N);
        ok = ok && dalloc(ctx, ctx->perm[b], N);
    }
    ok = ok && dalloc(ctx, ctx->patch_of, N);
    ok = ok && dalloc(ctx, ctx->keys, N) && dalloc(ctx, ctx->vals, N) && dalloc(ctx, ctx->keys_alt, N) &&
         dalloc(ctx, ctx->vals_alt, N);
    const size_t hw = radix_hist_words(ctx->cap_n);
    ok = ok && dalloc(ctx, ctx->hist, hw) && dalloc(ctx, ctx->scan32, (size_t)scan_tmp_words((int64_t)hw));
    uint4* cellrec = nullptr;
    uint32_t* cellxyz = nullptr;
    ok = ok && dalloc(ctx, cellrec, (size_t)ctx->cap_cells) && dalloc(ctx, cellxyz, N) &&
         dalloc(ctx, ctx->grid.hnb, (size_t)ctx->cap_cells) && dalloc(ctx, ctx->hnb_tmp, (size_t)ctx->cap_cells);
    ctx->grid.cell = cellrec;
    ctx->grid.cellxyz = cellxyz;
    // kGroup-style padding: the list search reads groups of records past a cell
    ok = ok && dalloc(ctx, ctx->rec.r4, N + 16);
    if (ctx->mixed) {
        ok = ok && dalloc(ctx, ctx->rec.r5, N) && dalloc(ctx, ctx->rec.rv, N) && dalloc(ctx, ctx->rec.rt, N) &&
             dalloc(ctx, ctx->rec.hc, N) && dalloc(ctx, ctx->rec.pf, N) && dalloc(ctx, ctx->rec.uf, N) &&
             dalloc(ctx, ctx->rec.acc, N);
    } else {
        Fp64& f = ctx->f64;
        double** g[14] = {&f.vhx, &f.vhy, &f.vhz, &f.rho, &f.P, &f.c, &f.A, &f.hc, &f.w, &f.w5, &f.ax, &f.ay, &f.az, &f.du};
        for (int k = 0; k < 14 && ok; k++) ok = dalloc(ctx, *g[k], N);
    }
    ok = ok && dalloc(ctx, ctx->bin_order, N) && dalloc(ctx, ctx->bin_bounds, (size_t)kPairOctaves + 1);
    ok = ok && dalloc(ctx, ctx->cnt, N) && dalloc(ctx, ctx->cnt_orig, N) && dalloc(ctx, ctx->nown, N) &&
         dalloc(ctx, ctx->off, N + 1) &&
         dalloc(ctx, ctx->col, (size_t)ctx->pool_cap) && dalloc(ctx, ctx->rowcap, N);
    ctx->cap_units = ctx->cap_n / 32 + ctx->cap_patch + 1;
    ok = ok && dalloc(ctx, ctx->rowstart, N) && dalloc(ctx, ctx->pool_used, 2) && dalloc(ctx, ctx->hint_ok, 1) &&
         dalloc(ctx, ctx->units, (size_t)ctx->cap_units) &&
         dalloc(ctx, ctx->scan64, (size_t)scan_tmp_words(ctx->cap_n));
    ok = ok && dalloc(ctx, ctx->pd, (size_t)ctx->cap_patch) && dalloc(ctx, ctx->red, (size_t)ctx->cap_patch) &&
         dalloc(ctx, ctx->items, (size_t)ctx->cap_items) && dalloc(ctx, ctx->partials, (size_t)ctx->cap_items * 7) &&
         dalloc(ctx, ctx->cons, (size_t)ctx->cap_patch * 7) && dalloc(ctx, ctx->scratch, N) &&
         dalloc(ctx, ctx->status, 1) && dalloc(ctx, ctx->pair_acc, 1) && dalloc(ctx, ctx->hfac, (size_t)kHFacN);
    if (ctx->skin > 0.0) {
        ok = ok && dalloc(ctx, ctx->col_s, (size_t)ctx->pool_cap) && dalloc(ctx, ctx->cnt_s, N) &&
             dalloc(ctx, ctx->hint_ok_s, 1) && dalloc(ctx, ctx->skinref.x0, N) && dalloc(ctx, ctx->skinref.y0, N) &&
             dalloc(ctx, ctx->skinref.z0, N) && dalloc(ctx, ctx->skinref.h0, N) && dalloc(ctx, ctx->skin_red, 2) &&
             dalloc(ctx, ctx->hsearch_pre, N) &&
             dalloc(ctx, ctx->skin_flag, 1);
        if (ok && cudaMallocHost(&ctx->h_skin_flag, sizeof(int)) != cudaSuccess) ok = false;
    }
    ctx->grid.patch_of = ctx->patch_of;
    ok = ok && dalloc(ctx, ctx->cf_vote, 2);
    if (ok && cudaMallocHost(&ctx->h_cf_vote, 2 * sizeof(unsigned long long)) != cudaSuccess) ok = false;
    if (ok && cudaMallocHost(&ctx->h_status, sizeof(int)) != cudaSuccess) ok = false;
    if (!ok) {
        sph_destroy(ctx);
        return fail(nullptr, SPH_ENOMEM, "device allocation failed for the requested capacities");
    }
    cudaMemsetAsync(ctx->status, 0, sizeof(int), ctx->stream);
    cudaMemsetAsync(ctx->pair_acc, 0, sizeof(unsigned long long), ctx->stream);
    {
        // R10: h <- h (1 + (n_target / n)^(1/3)) / 2, the factor for each count
        // below kHFacN in FP64 on the host
        std::vector<double> fac(kHFacN);
        fac[0] = 2.0;
        for (int k = 1; k < kHFacN; k++) fac[k] = 0.5 * (1.0 + std::cbrt(cfg.n_target / (double)k));
        if (cudaMemcpy(ctx->hfac, fac.data(), sizeof(double) * kHFacN, cudaMemcpyHostToDevice) != cudaSuccess) {
            sph_destroy(ctx);
            return fail(nullptr, SPH_ECUDA, "copy of the h-adaptation table failed");
        }
    }
    int64_t zero_off[2] = {0, 0};
    sph_status s = setup_patches(ctx, 1, zero_off);
    if (s != SPH_OK) {
        std::string m = ctx->err;
        sph_destroy(ctx);
        return fail(nullptr, s, m);
    }
    *out = ctx;
    return SPH_OK;
}

sph_status sph_set_particles(sph_ctx* ctx, int64_t n, const double* x, const double* y, const double* z,
                             const double* vx, const double* vy, const double* vz, const double* m,
                             const double* h, const double* u, int on_device)
{
    sph_status st = begin_call(ctx);
    if (st != SPH_OK) return st;
    if (n < 0 || n > ctx->cap_n) return fail(ctx, SPH_EINVAL, "n out of range [0, max_particles]");
    const double* src[9] = {x, y, z, vx, vy, vz, m, h, u};
    if (n > 0)
        for (int k = 0; k < 9; k++)
            if (!src[k]) return fail(ctx, SPH_EINVAL, "NULL field pointer");
    // the same number of particles again (one patch): the last lists' row
    // lengths, carried to the caller's order, reserve the rows of the first
    // search on the new particles (a set uploaded again keeps its rows; for
    // any other set they are only a poorer guess, which the search repairs)
    const bool carry = ctx->cnt_valid && n == ctx->n && n > 0 && ctx->npatch == 1;
    if (carry) {
        const int grid = (int)((n + 255) / 256 < ctx->sms * 16 ? (n + 255) / 256 : ctx->sms * 16);
        k_scatter_u32<<<grid, 256, 0, ctx->stream>>>(n, ctx->cnt, ctx->perm[ctx->cur], ctx->cnt_orig);
    }
    ctx->cur = 0;
    State& s = ctx->st[0];
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    for (int k = 0; k < 9; k++)
        if (n > 0) CK(cudaMemcpyAsync(state_field(s, k), src[k], (size_t)n * 8, kind, ctx->stream));
    for (int k = 9; k < 13; k++) CK(cudaMemsetAsync(state_field(s, k), 0, (size_t)(n > 0 ? n : 1) * 8, ctx->stream));
    ctx->n = n;
    if (n > 0) {
        const int grid = (int)((n + 255) / 256 < ctx->sms * 16 ? (n + 255) / 256 : ctx->sms * 16);
        k_iota<<<grid, 256, 0, ctx->stream>>>(n, ctx->perm[0]);
        launch_validate(launch_of(ctx), n, s, ctx->status);
    }
    int64_t offs[2] = {0, n};
    st = setup_patches(ctx, 1, offs);
    if (st != SPH_OK) return st;
    if (carry) {
        CK(cudaMemcpyAsync(ctx->cnt, ctx->cnt_orig, (size_t)n * sizeof(uint32_t), cudaMemcpyDeviceToDevice,
                           ctx->stream));
        CK(cudaMemsetAsync(ctx->hint_ok, 1, sizeof(int), ctx->stream));
        ctx->cnt_valid = true;
    }
    ctx->fresh = true;
    ctx->nnz = -1;
    st = check_status(ctx, "sph_set_particles");
    if (st == SPH_ENONFINITE)
        return fail(ctx, SPH_EINVAL, "sph_set_particles: inputs must be finite with m > 0 and h > 0");
    return st;
}

sph_status sph_set_patches(sph_ctx* ctx, int32_t n_patches, const int64_t* offsets)
{
    sph_status st = begin_call(ctx);
    if (st != SPH_OK) return st;
    if (!ctx->fresh) return fail(ctx, SPH_ESTATE, "sph_set_patches must follow sph_set_particles");
    if (n_patches < 1 || n_patches > ctx->cap_patch || !offsets)
        return fail(ctx, SPH_EINVAL, "n_patches out of range or offsets NULL");
    if (offsets[0] != 0 || offsets[n_patches] != ctx->n) return fail(ctx, SPH_EINVAL, "offsets must span [0, n]");
    for (int p = 0; p < n_patches; p++)
        if (offsets[p + 1] < offsets[p]) return fail(ctx, SPH_EINVAL, "offsets must be non-decreasing");
    return setup_patches(ctx, n_patches, offsets);
}

sph_status sph_find_neighbors(sph_ctx* ctx)
{
    sph_status st = begin_call(ctx);
    if (st != SPH_OK) return st;
    const bool reuse = reuse_lists(ctx);
    // with reused lists: the superset of the current order while it still
    // holds every pair (as a step would take it), else a fresh one
    const bool rebuild = !reuse || !ctx->sup_valid;
    ctx->nb_valid = ctx->rho_valid = ctx->acc_valid = false;
    ctx->sup_valid = ctx->sup_valid && reuse;
    if (rebuild) destroy_graphs(ctx);
    if (reuse) {
        if (rebuild) {
            enqueue_sort(ctx, true);
            enqueue_superset(ctx);
        }
        enqueue_filter(ctx);
    } else {
        enqueue_sort(ctx);
        enqueue_lists(ctx);
    }
    st = after_launches(ctx, "sph_find_neighbors");
    if (st != SPH_OK) return st;
    unsigned long long nnz = 0;
    CK(cudaMemcpyAsync(&nnz, ctx->pool_used + 1, sizeof(nnz), cudaMemcpyDeviceToHost, ctx->stream));
    st = check_status(ctx, "sph_find_neighbors");
    ctx->nnz = (int64_t)nnz;
    if (st != SPH_OK) return st;
    ctx->nb_valid = true;
    ctx->cnt_valid = true;
    if (reuse) {
        ctx->sup_valid = true;
        if (rebuild) ctx->rebuilds++;
    }
    return SPH_OK;
}

sph_status sph_get_neighbors(sph_ctx* ctx, const uint64_t** off, const uint32_t** col, const uint32_t** perm,
                             int64_t* nnz)
{
    sph_status st = begin_call(ctx);
    if (st != SPH_OK) return st;
    if (!ctx->nb_valid) return fail(ctx, SPH_ESTATE, "no current neighbour lists");
    if (!ctx->canon_valid) {
        // canonical CSR from the list pool: prefix offsets of the row lengths,
        // rows copied in particle order
        if (ctx->col_plain_cap < ctx->nnz) {
            if (ctx->col_plain) {
                for (auto& q : ctx->allocs)
                    if (q == (void*)ctx->col_plain) q = nullptr;
                cudaFree(ctx->col_plain);
                ctx->col_plain = nullptr;
                ctx->col_plain_cap = 0;
            }
            uint32_t* p = nullptr;
            if (!dalloc(ctx, p, (size_t)(ctx->nnz > 0 ? ctx->nnz : 1)))
                return fail(ctx, SPH_ENOMEM, "column buffer allocation failed");
            ctx->col_plain = p;
            ctx->col_plain_cap = ctx->nnz;
        }
        ctx->launches += launch_scan_u32_to_u64(launch_of(ctx), ctx->n, ctx->cnt, ctx->off, ctx->scan64);
        ctx->launches += launch_canonical_rows(launch_of(ctx), ctx->n, ctx->rowstart, ctx->cnt, ctx->off,
                                               ctx->col, ctx->col_plain);
        CK(cudaStreamSynchronize(ctx->stream));
        ctx->canon_valid = true;
    }
    if (col) *col = ctx->col_plain;
    if (off) *off = ctx->off;
    if (perm) *perm = ctx->perm[ctx->cur];
    if (nnz) *nnz = ctx->nnz;
    return after_launches(ctx, "sph_get_neighbors");
}

sph_status sph_copy_neighbors(sph_ctx* ctx, uint64_t* off, uint32_t* col, uint32_t* perm, int on_device)
{
    const uint64_t* o = nullptr;
    const uint32_t *c = nullptr, *pm = nullptr;
    int64_t nnz = 0;
    sph_status st = sph_get_neighbors(ctx, &o, col ? &c : nullptr, &pm, &nnz);
    if (st != SPH_OK) return st;
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (off) CK(cudaMemcpyAsync(off, o, sizeof(uint64_t) * (ctx->n + 1), k, ctx->stream));
    if (col && nnz > 0) CK(cudaMemcpyAsync(col, c, sizeof(uint32_t) * nnz, k, ctx->stream));
    if (perm && ctx->n > 0) CK(cudaMemcpyAsync(perm, pm, sizeof(uint32_t) * ctx->n, k, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return SPH_OK;
}

sph_status sph_density(sph_ctx* ctx)
{
    sph_status st = begin_call(ctx);
    if (st != SPH_OK) return st;
    if (!ctx->nb_valid)
        return fail(ctx, SPH_ESTATE, "sph_density needs sph_find_neighbors on the current particles");
    enqueue_density(ctx);
    st = after_launches(ctx, "sph_density");
    if (st != SPH_OK) return st;
    st = check_status(ctx, "sph_density");
    ctx->rho_valid = st == SPH_OK;
    ctx->acc_valid = false;
    return st;
}

sph_status sph_momentum_energy(sph_ctx* ctx)
{
    sph_status st = begin_call(ctx);
    if (st != SPH_OK) return st;
    if (!ctx->rho_valid) return fail(ctx, SPH_ESTATE, "sph_momentum_energy needs sph_density first");
    enqueue_momentum(ctx);
    st = after_launches(ctx, "sph_momentum_energy");
    if (st != SPH_OK) return st;
    st = check_status(ctx, "sph_momentum_energy");
    ctx->acc_valid = st == SPH_OK;
    return st;
}

sph_status sph_step(sph_ctx* ctx, int32_t nsteps, double* dt_last)
{
    sph_status st = begin_call(ctx);
    if (st != SPH_OK) return st;
    if (nsteps < 0) return fail(ctx, SPH_EINVAL, "nsteps < 0");
    if (ctx->n == 0) return SPH_OK;
    const bool graph = ctx->cfg.use_graph && !ctx->prof;
    const bool reuse = reuse_lists(ctx);
    for (int k = 0; k < nsteps; k++) {
        // with reused lists: sort and search only when the superset no longer
        // holds every pair (the previous step's check says so)
        const bool rebuild = !reuse || !ctx->sup_valid;
        // the first step after new particles runs outside the graphs: a
        // captured step must not depend on the state having no search yet
        if (graph && !ctx->fresh) {
            const int par = ctx->cur, kind = rebuild ? 1 : 0;
            if (!ctx->gexec[par][kind]) {
                cudaGraph_t g = nullptr;
                const int64_t l0 = ctx->launches;
                CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
                enqueue_step(ctx, rebuild);
                cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
                ctx->cur = par;
                ctx->launches = l0;
                if (e != cudaSuccess) return cuda_fail(ctx, e, "graph capture");
                int64_t nk = 0;
                size_t nn = 0;
                cudaGraphGetNodes(g, nullptr, &nn);
                std::vector<cudaGraphNode_t> nodes(nn);
                cudaGraphGetNodes(g, nodes.data(), &nn);
                for (auto nd : nodes) {
                    cudaGraphNodeType ty;
                    cudaGraphNodeGetType(nd, &ty);
                    if (ty == cudaGraphNodeTypeKernel) nk++;
                }
                e = cudaGraphInstantiate(&ctx->gexec[par][kind], g, 0);
                cudaGraphDestroy(g);
                if (e != cudaSuccess) return cuda_fail(ctx, e, "graph instantiate");
                ctx->graph_kernels[par][kind] = nk;
            }
            CK(cudaGraphLaunch(ctx->gexec[par][kind], ctx->stream));
            ctx->launches += ctx->graph_kernels[par][kind];
            // a step with a sort moves the state to the other buffer
            ctx->cur = rebuild ? 1 - par : par;
            ctx->fresh = false;
        } else {
            enqueue_step(ctx, rebuild);
        }
        if (reuse) {
            CK(cudaMemcpyAsync(ctx->h_skin_flag, ctx->skin_flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
            CK(cudaStreamSynchronize(ctx->stream));
            ctx->sup_valid = *ctx->h_skin_flag != 0;
            if (rebuild) ctx->rebuilds++;
        }
    }
    st = after_launches(ctx, "sph_step");
    if (st != SPH_OK) return st;
    st = check_status(ctx, "sph_step");
    ctx->nb_valid = false;
    ctx->rho_valid = ctx->acc_valid = (st == SPH_OK);
    ctx->cnt_valid = st == SPH_OK;
    if (st != SPH_OK) return st;
    if (dt_last) {
        CK(cudaMemcpy(dt_last, &ctx->pd[0].dt, sizeof(double), cudaMemcpyDeviceToHost));
    }
    // an automatic cell factor of 1/2 or 0.4 follows the vote of the last
    // sort: the 3-cell stencil over median-sized cells (0.4) once most
    // non-empty cells of patches with a wide spread of h see no h above
    // 0.8 h_s around them, cells of edge h_s (1/2) again when few do.  The
    // vote depends on the state alone, so a run is reproducible for a given
    // sequence of calls; the new grid takes effect at the next call.
    if (ctx->cf_auto && (ctx->cell_factor == 0.4 || ctx->cell_factor == 0.5)) {
        CK(cudaMemcpy(ctx->h_cf_vote, ctx->cf_vote, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
        const unsigned long long ne = ctx->h_cf_vote[0], nn = ctx->h_cf_vote[1];
        double want = ctx->cell_factor;
        if (ctx->cell_factor == 0.5 && nn * 20 > ne * 11) want = 0.4;        // above 55 %
        else if (ctx->cell_factor == 0.4 && nn * 10 < ne * 3) want = 0.5;    // below 30 %
        if (want != ctx->cell_factor) {
            ctx->cell_factor = want;
            ctx->cf_switches++;
            destroy_graphs(ctx);
        }
    }
    return SPH_OK;
}

sph_status sph_conserved(sph_ctx* ctx, int32_t patch, double out[7])
{
    sph_status st = begin_call(ctx);
    if (st != SPH_OK) return st;
    if (!out || patch < -1 || patch >= ctx->npatch) return fail(ctx, SPH_EINVAL, "bad patch or out");
    const StepArgs a = step_args(ctx);
    ctx->launches += launch_conserved_items(launch_of(ctx), a);
    ctx->launches += launch_conserved_finalize(launch_of(ctx), a);
    st = after_launches(ctx, "sph_conserved");
    if (st != SPH_OK) return st;
    std::vector<double> c((size_t)ctx->npatch * 7);
    CK(cudaMemcpyAsync(c.data(), ctx->cons, sizeof(double) * c.size(), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (patch >= 0) {
        for (int q = 0; q < 7; q++) out[q] = c[(size_t)patch * 7 + q];
    } else {
        for (int q = 0; q < 7; q++) {
            double s = 0.0, comp = 0.0;
            for (int p = 0; p < ctx->npatch; p++) {
                const double v = c[(size_t)p * 7 + q];
                const double t = s + v;
                if (fabs(s) >= fabs(v)) comp += (s - t) + v;
                else comp += (v - t) + s;
                s = t;
            }
            out[q] = s + comp;
        }
    }
    return SPH_OK;
}

sph_status sph_get_field(sph_ctx* ctx, int32_t field, double* dst, int on_device)
{
    sph_status st = begin_call(ctx);
    if (st != SPH_OK) return st;
    if (field < 0 || field >= SPH_FIELD_COUNT) return fail(ctx, SPH_EINVAL, "unknown field");
    if (!dst && ctx->n > 0) return fail(ctx, SPH_EINVAL, "dst is NULL");
    if (ctx->n == 0) return SPH_OK;
    const Launch L = launch_of(ctx);
    double* out = on_device ? dst : ctx->scratch;
    const uint32_t* perm = ctx->perm[ctx->cur];
    const int64_t n = ctx->n;
    if (field <= SPH_FIELD_AZP) {
        ctx->launches += launch_unpermute_f64(L, n, state_field(ctx->st[ctx->cur], field), perm, out);
    } else if (field <= SPH_FIELD_C) {
        if (!ctx->rho_valid) return fail(ctx, SPH_ESTATE, "density not computed for the current order");
        if (ctx->mixed) {
            if (field == SPH_FIELD_P) ctx->launches += launch_unpermute_f32(L, n, ctx->rec.pf, 1, perm, out);
            else ctx->launches += launch_unpermute_f32(L, n, (const float*)ctx->rec.rt + (field == SPH_FIELD_RHO ? 0 : 2),
                                                       4, perm, out);
        } else {
            const double* s = field == SPH_FIELD_RHO ? ctx->f64.rho : (field == SPH_FIELD_P ? ctx->f64.P : ctx->f64.c);
            ctx->launches += launch_unpermute_f64(L, n, s, perm, out);
        }
    } else if (field <= SPH_FIELD_DU) {
        if (!ctx->acc_valid) return fail(ctx, SPH_ESTATE, "accelerations not computed for the current order");
        const int k = field - SPH_FIELD_AX;
        if (ctx->mixed) {
            ctx->launches += launch_unpermute_f32(L, n, (const float*)ctx->rec.acc + k, 4, perm, out);
        } else {
            const double* s[4] = {ctx->f64.ax, ctx->f64.ay, ctx->f64.az, ctx->f64.du};
            ctx->launches += launch_unpermute_f64(L, n, s[k], perm, out);
        }
    } else if (field == SPH_FIELD_NOWN) {
        if (ctx->fresh) return fail(ctx, SPH_ESTATE, "no neighbour search yet");
        ctx->launches += launch_unpermute_u32(L, n, ctx->nown, perm, out);
    } else {
        if (ctx->fresh) return fail(ctx, SPH_ESTATE, "no neighbour search yet");
        ctx->launches += launch_unpermute_u32(L, n, ctx->cnt, perm, out);
    }
    st = after_launches(ctx, "sph_get_field");
    if (st != SPH_OK) return st;
    if (!on_device) CK(cudaMemcpyAsync(dst, out, (size_t)n * 8, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return SPH_OK;
}

sph_status sph_get_dt(sph_ctx* ctx, int32_t patch, double* dt, double* dt_prev, int64_t* step)
{
    sph_status st = begin_call(ctx);
    if (st != SPH_OK) return st;
    if (patch < 0 || patch >= ctx->npatch) return fail(ctx, SPH_EINVAL, "bad patch");
    PatchDev P;
    CK(cudaMemcpyAsync(&P, ctx->pd + patch, sizeof(P), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (dt) *dt = P.dt;
    if (dt_prev) *dt_prev = P.dt_prev;
    if (step) *step = P.step;
    return SPH_OK;
}

namespace {
struct StateHeader {
    char magic[8];
    int64_t version, n, npatch, reserved;
};
}  // namespace

sph_status sph_get_state(sph_ctx* ctx, void* buf, size_t* bytes)
{
    sph_status st = begin_call(ctx);
    if (st != SPH_OK) return st;
    if (!bytes) return fail(ctx, SPH_EINVAL, "bytes is NULL");
    const int64_t n = ctx->n, np = ctx->npatch;
    const size_t need = sizeof(StateHeader) + sizeof(int64_t) * (np + 1) + sizeof(double) * 3 * np +
                        sizeof(uint32_t) * n + sizeof(double) * 13 * n;
    if (!buf) {
        *bytes = need;
        return SPH_OK;
    }
    if (*bytes < need) return fail(ctx, SPH_EINVAL, "buffer too small");
    char* p = (char*)buf;
    StateHeader h;
    memcpy(h.magic, "SPHGB300", 8);
    h.version = 1;
    h.n = n;
    h.npatch = np;
    h.reserved = 0;
    memcpy(p, &h, sizeof(h));
    p += sizeof(h);
    memcpy(p, ctx->patch_off.data(), sizeof(int64_t) * (np + 1));
    p += sizeof(int64_t) * (np + 1);
    std::vector<PatchDev> pd(np);
    CK(cudaMemcpyAsync(pd.data(), ctx->pd, sizeof(PatchDev) * np, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int q = 0; q < np; q++) {
        double t[3] = {pd[q].dt, pd[q].dt_prev, (double)pd[q].step};
        memcpy(p, t, sizeof(t));
        p += sizeof(t);
    }
    if (n > 0) {
        CK(cudaMemcpy(p, ctx->perm[ctx->cur], sizeof(uint32_t) * n, cudaMemcpyDeviceToHost));
        p += sizeof(uint32_t) * n;
        for (int k = 0; k < 13; k++) {
            CK(cudaMemcpy(p, state_field(ctx->st[ctx->cur], k), sizeof(double) * n, cudaMemcpyDeviceToHost));
            p += sizeof(double) * n;
        }
    }
    *bytes = need;
    return SPH_OK;
}

sph_status sph_set_state(sph_ctx* ctx, const void* buf, size_t bytes)
{
    sph_status st = begin_call(ctx);
    if (st != SPH_OK) return st;
    if (!buf || bytes < sizeof(StateHeader)) return fail(ctx, SPH_EINVAL, "bad state buffer");
    const char* p = (const char*)buf;
    StateHeader h;
    memcpy(&h, p, sizeof(h));
    p += sizeof(h);
    if (memcmp(h.magic, "SPHGB300", 8) != 0 || h.version != 1) return fail(ctx, SPH_EINVAL, "not a state buffer");
    const int64_t n = h.n, np = h.npatch;
    if (n < 0 || n > ctx->cap_n || np < 1 || np > ctx->cap_patch) return fail(ctx, SPH_EINVAL, "state exceeds capacity");
    const size_t need = sizeof(StateHeader) + sizeof(int64_t) * (np + 1) + sizeof(double) * 3 * np +
                        sizeof(uint32_t) * n + sizeof(double) * 13 * n;
    if (bytes < need) return fail(ctx, SPH_EINVAL, "state buffer truncated");
    std::vector<int64_t> offs(np + 1);
    memcpy(offs.data(), p, sizeof(int64_t) * (np + 1));
    p += sizeof(int64_t) * (np + 1);
    std::vector<double> times(3 * np);
    memcpy(times.data(), p, sizeof(double) * 3 * np);
    p += sizeof(double) * 3 * np;
    // as in sph_set_particles: the last lists' row lengths, carried to the
    // caller's order and then into the restored state's order, reserve the
    // rows of its first search (a state saved by this context a step ago
    // gets its own rows back; any other hint is only a poorer guess)
    const bool carry = ctx->cnt_valid && n == ctx->n && n > 0;
    const int cgrid = (int)((n + 255) / 256 < ctx->sms * 16 ? (n + 255) / 256 : ctx->sms * 16);
    if (carry) k_scatter_u32<<<cgrid, 256, 0, ctx->stream>>>(n, ctx->cnt, ctx->perm[ctx->cur], ctx->cnt_orig);
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->cur = 0;
    ctx->n = n;
    if (n > 0) {
        CK(cudaMemcpy(ctx->perm[0], p, sizeof(uint32_t) * n, cudaMemcpyHostToDevice));
        p += sizeof(uint32_t) * n;
        for (int k = 0; k < 13; k++) {
            CK(cudaMemcpy(state_field(ctx->st[0], k), p, sizeof(double) * n, cudaMemcpyHostToDevice));
            p += sizeof(double) * n;
        }
    }
    st = setup_patches(ctx, (int)np, offs.data());
    if (st != SPH_OK) return st;
    std::vector<PatchDev> pd(np);
    CK(cudaMemcpy(pd.data(), ctx->pd, sizeof(PatchDev) * np, cudaMemcpyDeviceToHost));
    for (int q = 0; q < np; q++) {
        pd[q].dt = times[3 * q];
        pd[q].dt_prev = times[3 * q + 1];
        pd[q].step = (int64_t)times[3 * q + 2];
    }
    CK(cudaMemcpy(ctx->pd, pd.data(), sizeof(PatchDev) * np, cudaMemcpyHostToDevice));
    if (carry) {
        k_gather_u32<<<cgrid, 256, 0, ctx->stream>>>(n, ctx->cnt_orig, ctx->perm[0], ctx->cnt);
        CK(cudaMemsetAsync(ctx->hint_ok, 1, sizeof(int), ctx->stream));
        ctx->cnt_valid = true;
        st = after_launches(ctx, "sph_set_state");
        if (st != SPH_OK) return st;
    }
    ctx->fresh = true;
    ctx->nnz = -1;
    return SPH_OK;
}

sph_status sph_autotune(sph_ctx* ctx)
{
    sph_status st = begin_call(ctx);
    if (st != SPH_OK) return st;
    if (ctx->n == 0) return SPH_OK;
    const bool prof0 = ctx->prof;
    ctx->prof = false;
    destroy_graphs(ctx);
    // 1/3 and 0.4 (a 3-cell stencil) take cells down to min(h_s, 1.3 h_median)
    const double factors[5] = {1.0 / 3.0, 0.4, 0.5, 0.75, 1.0};
    const int pair_tpps[6] = {1, 2, 4, 8, 16, 32};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto timeit = [&](auto&& fn) {
        float best = 1e30f;
        for (int rep = 0; rep < 2; rep++) {
            cudaEventRecord(e0, ctx->stream);
            fn();
            cudaEventRecord(e1, ctx->stream);
            cudaEventSynchronize(e1);
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) best = ms;
        }
        return best;
    };
    // lists: the search writing them plus the best launch shape of each sum
    // over them (a uniform lanes-per-particle count, or row-length bins with
    // a words-per-lane target, whose binning pass is paid once per step);
    // list-free: the two passes (each runs the search)
    const bool try_lists = ctx->cfg.pair_mode != SPH_PAIRS_FUSED;
    const bool try_fused = ctx->cfg.pair_mode != SPH_PAIRS_LISTS;
    const bool fixed_bins = ctx->cfg.pair_bins > 0;
    const bool try_bins = ctx->cfg.pair_bins == 0;
    const int bin_ws[4] = {4, 5, 6, 7};   // 16 .. 128 list words per lane
    double best_total = 1e300, best_f = ctx->cell_factor;
    int best_pair = ctx->tpp_pair, best_den = ctx->tpp_den;
    int best_bpair = ctx->bins_pair, best_bden = ctx->bins_den;
    bool best_fused = ctx->fused;
    for (double f : factors) {
        ctx->cell_factor = f;
        enqueue_sort(ctx);
        if (try_lists) {
            ctx->fused = false;
            const float bnb = timeit([&] { enqueue_lists(ctx); });
            // uniform shapes
            float uden = 1e30f, umom = 1e30f, bden = 1e30f, bmom = 1e30f;
            int tden = 8, tmom = 8, wden = 0, wmom = 0;
            if (!fixed_bins) {
                ctx->bins_den = ctx->bins_pair = 0;
                for (int t : pair_tpps) {
                    ctx->tpp_den = t;
                    const float ms = timeit([&] { enqueue_density(ctx); });
                    if (ms < uden) { uden = ms; tden = t; }
                }
            }
            float tbin = 0.0f;
            if (try_bins || fixed_bins) {
                tbin = timeit([&] { ctx->bins_valid = false; enqueue_bins(ctx); });
                for (int w : bin_ws) {
                    if (fixed_bins && w != ctx->bins_den) continue;
                    ctx->bins_den = w;
                    const float ms = timeit([&] { enqueue_density(ctx); });
                    if (ms < bden) { bden = ms; wden = w; }
                }
                if (fixed_bins) wden = ctx->bins_den;
            }
            // the momentum sum reads the density's records: one density sum first
            ctx->bins_den = 0;
            ctx->tpp_den = tden;
            enqueue_density(ctx);
            if (!fixed_bins) {
                ctx->bins_pair = 0;
                for (int t : pair_tpps) {
                    ctx->tpp_pair = t;
                    const float ms = timeit([&] { enqueue_momentum(ctx); });
                    if (ms < umom) { umom = ms; tmom = t; }
                }
            }
            if (try_bins || fixed_bins) {
                for (int w : bin_ws) {
                    if (fixed_bins && w != ctx->bins_pair) continue;
                    ctx->bins_pair = w;
                    const float ms = timeit([&] { enqueue_momentum(ctx); });
                    if (ms < bmom) { bmom = ms; wmom = w; }
                }
            }
            // the four combinations of uniform and binned sums
            for (int c = 0; c < 4; c++) {
                const bool bd = c & 1, bm = c & 2;
                if ((bd && !wden) || (bm && !wmom) || (!bd && uden >= 1e29f) || (!bm && umom >= 1e29f)) continue;
                const double tot = (double)bnb + (bd ? bden : uden) + (bm ? bmom : umom) + ((bd || bm) ? tbin : 0.0f);
                if (tot < best_total) {
                    best_total = tot;
                    best_f = f;
                    best_den = tden;
                    best_pair = tmom;
                    best_bden = bd ? wden : 0;
                    best_bpair = bm ? wmom : 0;
                    best_fused = false;
                }
            }
        }
        if (try_fused) {
            ctx->fused = true;
            const double tot = timeit([&] { enqueue_density(ctx); enqueue_momentum(ctx); });
            if (tot < best_total) {
                best_total = tot;
                best_f = f;
                best_fused = true;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->cell_factor = best_f;
    ctx->cf_auto = true;
    ctx->tpp_pair = best_pair;
    ctx->tpp_den = best_den;
    ctx->bins_pair = best_bpair;
    ctx->bins_den = best_bden;
    ctx->bins_valid = false;
    ctx->fused = best_fused;
    ctx->prof = prof0;
    ctx->nb_valid = ctx->rho_valid = ctx->acc_valid = ctx->sup_valid = false;
    st = after_launches(ctx, "sph_autotune");
    if (st != SPH_OK) return st;
    st = check_status(ctx, "sph_autotune");
    ctx->cnt_valid = st == SPH_OK;   // the last timed search's rows, in the current order
    return st;
}

sph_status sph_get_tuning(sph_ctx* ctx, int32_t* tpp, double* cell_factor)
{
    if (!ctx) return fail(nullptr, SPH_EINVAL, "null context");
    if (tpp) *tpp = ctx->tpp_pair;
    if (cell_factor) *cell_factor = ctx->cell_factor;
    return SPH_OK;
}

sph_status sph_get_density_tpp(sph_ctx* ctx, int32_t* tpp)
{
    if (!ctx) return fail(nullptr, SPH_EINVAL, "null context");
    if (tpp) *tpp = ctx->tpp_den;
    return SPH_OK;
}

sph_status sph_get_pair_bins(sph_ctx* ctx, int32_t* words_density, int32_t* words_momentum)
{
    if (!ctx) return fail(nullptr, SPH_EINVAL, "null context");
    if (words_density) *words_density = ctx->bins_den ? 1 << ctx->bins_den : 0;
    if (words_momentum) *words_momentum = ctx->bins_pair ? 1 << ctx->bins_pair : 0;
    return SPH_OK;
}

sph_status sph_get_pair_mode(sph_ctx* ctx, int32_t* mode)
{
    if (!ctx) return fail(nullptr, SPH_EINVAL, "ctx is NULL");
    if (mode) *mode = ctx->fused ? SPH_PAIRS_FUSED : SPH_PAIRS_LISTS;
    return SPH_OK;
}

sph_status sph_get_list_rebuilds(sph_ctx* ctx, int64_t* n)
{
    if (!ctx) return fail(nullptr, SPH_EINVAL, "null context");
    if (n) *n = ctx->rebuilds;
    return SPH_OK;
}

sph_status sph_set_profiling(sph_ctx* ctx, int enable)
{
    if (!ctx) return fail(nullptr, SPH_EINVAL, "null context");
    ctx->prof = enable != 0;
    return SPH_OK;
}

sph_status sph_get_profile(sph_ctx* ctx, double* ms, int64_t* launches, int32_t nphase)
{
    if (!ctx) return fail(nullptr, SPH_EINVAL, "null context");
    collect_profile(ctx);
    for (int k = 0; k < nphase && k < SPH_PHASE_COUNT; k++) {
        if (ms) ms[k] = ctx->prof_ms[k];
        if (launches) launches[k] = ctx->prof_launch[k];
    }
    for (int k = 0; k < SPH_PHASE_COUNT; k++) {
        ctx->prof_ms[k] = 0.0;
        ctx->prof_launch[k] = 0;
    }
    return SPH_OK;
}

sph_status sph_get_launch_count(sph_ctx* ctx, int64_t* launches)
{
    if (!ctx || !launches) return fail(ctx, SPH_EINVAL, "null argument");
    *launches = ctx->launches;
    return SPH_OK;
}

sph_status sph_get_pair_count(sph_ctx* ctx, int64_t* total, int reset)
{
    if (!ctx || !total) return fail(ctx, SPH_EINVAL, "null argument");
    unsigned long long v = 0;
    CK(cudaMemcpyAsync(&v, ctx->pair_acc, sizeof(v), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    *total = (int64_t)v;
    if (reset) CK(cudaMemsetAsync(ctx->pair_acc, 0, sizeof(v), ctx->stream));
    return SPH_OK;
}

sph_status sph_get_nnz(sph_ctx* ctx, int64_t* nnz)
{
    if (!ctx || !nnz) return fail(ctx, SPH_EINVAL, "null argument");
    *nnz = ctx->nnz;
    return SPH_OK;
}

}  // extern "C"
