// sph_step.cu -- the rest of the timestep (Sec. 3), all in FP64:
//   Courant condition, global per patch (R7):
//       dt_n = min(C min_i h_i / c_i, dt_growth dt_{n-1})      (dt_0 without cap)
//   Press / leapfrog positions (R8):
//       v_{n+1/2} = v_{n-1/2} + a_n (dt_n + dt_{n-1}) / 2      (dt_{-1} := 0)
//       x_{n+1}   = x_n + v_{n+1/2} dt_n, z wrapped into [-lz/2, lz/2)
//   Adams-Bashforth energy (R8):
//       u_{n+1} = u_n + dt_n [(1 + r/2) du_n - (r/2) du_{n-1}], r = dt_n/dt_{n-1}
//       (Euler on the first step)
//   smoothing length (R10): h <- h (1 + (N_t / n_i)^(1/3)) / 2, doubled if n_i = 0
//   conserved sums (Sec. 4 stresses conservation laws): M, P, L_z, E_kin, E_int,
//       per work item in a fixed-shape block reduction, then per patch in item
//       order with compensation -- deterministic.
#include "sph_internal.cuh"

namespace sphg {

__device__ __forceinline__ double warp_sum_d(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// sum of 7 per-thread values over a block of 256 threads; result valid in thread 0
__device__ __forceinline__ void block_sum7(double v[7], double (*sh)[8])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = 0; q < 7; q++) v[q] = warp_sum_d(v[q]);
    if (lane == 0)
        for (int q = 0; q < 7; q++) sh[q][warp] = v[q];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 0; q < 7; q++) {
            double s = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += sh[q][w];
            v[q] = s;
        }
    }
    __syncthreads();
}

// one particle's share of the conserved sums, accumulated with FMAs: M, P,
// L_z = m (x v_y - y v_x), twice E_kin (halved once per work item), E_int
__device__ __forceinline__ void cons_accum(double x, double y, double vx, double vy, double vz, double m,
                                           double u, double acc[7])
{
    acc[0] += m;
    acc[1] = fma(m, vx, acc[1]);
    acc[2] = fma(m, vy, acc[2]);
    acc[3] = fma(m, vz, acc[3]);
    acc[4] = fma(m, fma(x, vy, -y * vx), acc[4]);
    acc[5] = fma(m, fma(vx, vx, fma(vy, vy, vz * vz)), acc[5]);
    acc[6] = fma(m, u, acc[6]);
}

// ---- min over particles of h/c, per patch ---------------------------------
__global__ void __launch_bounds__(256) k_hc_min(StepArgs a)
{
    __shared__ unsigned long long sh[8];
    if (*a.status & kStBad) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int it = blockIdx.x; it < a.nitems; it += gridDim.x) {
        const WorkItem w = a.items[it];
        unsigned long long mn = ~0ull;
        for (int64_t i = w.begin + threadIdx.x; i < w.end; i += blockDim.x) {
            const double v = a.mixed ? (double)a.r.hc[i] : a.f.hc[i];
            const unsigned long long o = ord_f64(v);
            mn = o < mn ? o : mn;
        }
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long t = __shfl_xor_sync(0xffffffffu, mn, o);
            mn = t < mn ? t : mn;
        }
        if (lane == 0) sh[warp] = mn;
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int ww = 1; ww < (int)(blockDim.x >> 5); ww++) mn = sh[ww] < mn ? sh[ww] : mn;
            atomicMin(&a.red[w.patch].hcmin, mn);
        }
        __syncthreads();
    }
}

// every step starts its minima afresh (a step that reuses its lists runs no
// sort, whose reset would otherwise clear them)
__global__ void k_hc_reset(PatchRed* red, int npatch)
{
    for (int p = threadIdx.x; p < npatch; p += blockDim.x) red[p].hcmin = ~0ull;
}

int launch_hc_min(const Launch& L, const StepArgs& a)
{
    if (a.nitems <= 0) return 0;
    k_hc_reset<<<1, 256, 0, L.stream>>>(a.red, a.npatch);
    const int grid = a.nitems < L.sms * 8 ? a.nitems : L.sms * 8;
    k_hc_min<<<grid, 256, 0, L.stream>>>(a);
    return 2;
}

// ---- Courant time-step per patch ------------------------------------------
__global__ void k_dt(StepArgs a)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.npatch || (*a.status & kStBad)) return;
    PatchDev* P = a.pd + p;
    if (P->end <= P->begin) {
        P->dt = 0.0;
        return;
    }
    double dt;
    if (a.dt_fixed > 0.0) {
        dt = a.dt_fixed;
    } else {
        dt = a.courant * unord_f64(a.red[p].hcmin);
        if (P->step > 0 && a.dt_growth * P->dt_prev < dt) dt = a.dt_growth * P->dt_prev;
    }
    if (!(dt > 0.0) || !isfinite(dt)) atomicOr(a.status, kStNonFinite);
    P->dt = dt;
}

int launch_dt(const Launch& L, const StepArgs& a)
{
    k_dt<<<(a.npatch + 127) / 128, 128, 0, L.stream>>>(a);
    return 1;
}

// ---- kick, drift, Adams-Bashforth, h, conserved partials --------------------
__global__ void __launch_bounds__(256) k_update(StepArgs a)
{
    __shared__ double sh[7][8];
    if (*a.status & kStBad) return;
    for (int it = blockIdx.x; it < a.nitems; it += gridDim.x) {
        const WorkItem w = a.items[it];
        const PatchDev* P = a.pd + w.patch;
        const double dt = P->dt, lz = P->lz;
        const bool first = P->step == 0;
        const double kick = 0.5 * (dt + (first ? 0.0 : P->dt_prev));
        const double r = first ? 0.0 : dt / P->dt_prev;
        const double c1 = 1.0 + 0.5 * r, c0 = 0.5 * r;
        double acc[7] = {0, 0, 0, 0, 0, 0, 0};
        for (int64_t i = w.begin + threadIdx.x; i < w.end; i += blockDim.x) {
            double ax, ay, az, du;
            if (a.mixed) {
                const float4 q = a.r.acc[i];
                ax = q.x; ay = q.y; az = q.z; du = q.w;
            } else {
                ax = a.f.ax[i]; ay = a.f.ay[i]; az = a.f.az[i]; du = a.f.du[i];
            }
            const double vx = a.s.vx[i] + ax * kick;
            const double vy = a.s.vy[i] + ay * kick;
            const double vz = a.s.vz[i] + az * kick;
            const double x = a.s.x[i] + vx * dt;
            const double y = a.s.y[i] + vy * dt;
            double z = a.s.z[i] + vz * dt;
            if (z >= 0.5 * lz) z -= lz;
            else if (z < -0.5 * lz) z += lz;
            const double u0 = a.s.u[i];
            const double u = first ? u0 + dt * du : u0 + dt * (c1 * du - c0 * a.s.du_prev[i]);
            a.s.vx[i] = vx; a.s.vy[i] = vy; a.s.vz[i] = vz;
            a.s.x[i] = x; a.s.y[i] = y; a.s.z[i] = z;
            a.s.u[i] = u;
            a.s.du_prev[i] = du;
            a.s.axp[i] = ax; a.s.ayp[i] = ay; a.s.azp[i] = az;
            if (a.adapt_h) {
                // R10 factor: a table of the host's FP64 values for the usual
                // counts, the same expression on the device beyond it
                const uint32_t ni = a.nown[i];
                double f;
                if (ni == 0) f = 2.0;
                else if (ni < (uint32_t)kHFacN) f = a.hfac[ni];
                else f = 0.5 * (1.0 + cbrt(a.n_target / (double)ni));
                a.s.h[i] *= f;
            }
            cons_accum(x, y, vx, vy, vz, a.s.m[i], u, acc);
        }
        acc[5] *= 0.5;
        block_sum7(acc, sh);
        if (threadIdx.x == 0)
            for (int q = 0; q < 7; q++) a.partials[(int64_t)it * 7 + q] = acc[q];
    }
}

int launch_update(const Launch& L, const StepArgs& a)
{
    if (a.nitems <= 0) return 0;
    const int grid = a.nitems < L.sms * 8 ? a.nitems : L.sms * 8;
    k_update<<<grid, 256, 0, L.stream>>>(a);
    return 1;
}

__global__ void __launch_bounds__(256) k_conserved_items(StepArgs a)
{
    __shared__ double sh[7][8];
    for (int it = blockIdx.x; it < a.nitems; it += gridDim.x) {
        const WorkItem w = a.items[it];
        double acc[7] = {0, 0, 0, 0, 0, 0, 0};
        for (int64_t i = w.begin + threadIdx.x; i < w.end; i += blockDim.x)
            cons_accum(a.s.x[i], a.s.y[i], a.s.vx[i], a.s.vy[i], a.s.vz[i], a.s.m[i], a.s.u[i], acc);
        acc[5] *= 0.5;
        block_sum7(acc, sh);
        if (threadIdx.x == 0)
            for (int q = 0; q < 7; q++) a.partials[(int64_t)it * 7 + q] = acc[q];
    }
}

int launch_conserved_items(const Launch& L, const StepArgs& a)
{
    if (a.nitems <= 0) return 0;
    const int grid = a.nitems < L.sms * 8 ? a.nitems : L.sms * 8;
    k_conserved_items<<<grid, 256, 0, L.stream>>>(a);
    return 1;
}

__device__ __forceinline__ void neumaier_add(double& s, double& c, double v)
{
    const double t = s + v;
    if (fabs(s) >= fabs(v)) c += (s - t) + v;
    else c += (v - t) + s;
    s = t;
}

// one warp per (patch, quantity): lane l takes the item partials l, l + 32,
// ... in order with a compensated sum; lane 0 then adds the 32 lane sums in
// lane order.  The order is fixed, so the result is reproducible.  With
// advance != 0 (after an update) it also closes the step.
__global__ void __launch_bounds__(32) k_conserved_finalize(StepArgs a, int advance)
{
    const int t = blockIdx.x;
    if (t >= a.npatch * 7) return;
    const int lane = threadIdx.x;
    const int p = t / 7, q = t % 7;
    PatchDev* P = a.pd + p;
    const bool ok = !(*a.status & kStBad);
    if (advance && !ok) return;
    double s = 0.0, c = 0.0;
    for (int it = P->item_begin + lane; it < P->item_end; it += 32)
        neumaier_add(s, c, a.partials[(int64_t)it * 7 + q]);
    double S = 0.0, C = 0.0;
    for (int l = 0; l < 32; l++) {
        const double sl = __shfl_sync(0xffffffffu, s, l);
        const double cl = __shfl_sync(0xffffffffu, c, l);
        neumaier_add(S, C, sl);
        C += cl;
    }
    if (lane == 0) {
        a.cons[p * 7 + q] = S + C;
        if (advance && q == 0) {
            P->dt_prev = P->dt;
            P->step += 1;
        }
    }
}

int launch_conserved_finalize(const Launch& L, const StepArgs& a)
{
    k_conserved_finalize<<<a.npatch * 7, 32, 0, L.stream>>>(a, 0);
    return 1;
}

int launch_step_finalize(const Launch& L, const StepArgs& a)
{
    k_conserved_finalize<<<a.npatch * 7, 32, 0, L.stream>>>(a, 1);
    return 1;
}

// ---- helpers for the ABI ---------------------------------------------------
static inline unsigned grid_n(const Launch& L, int64_t n)
{
    int64_t b = (n + 255) / 256;
    if (b > (int64_t)L.sms * 16) b = (int64_t)L.sms * 16;
    return (unsigned)(b < 1 ? 1 : b);
}

__global__ void k_unpermute_f64(int64_t n, const double* src, const uint32_t* perm, double* dst)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        dst[perm[k]] = src[k];
}
__global__ void k_unpermute_f32(int64_t n, const float* src, int stride, const uint32_t* perm, double* dst)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        dst[perm[k]] = (double)src[k * stride];
}
__global__ void k_unpermute_u32(int64_t n, const uint32_t* src, const uint32_t* perm, double* dst)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        dst[perm[k]] = (double)src[k];
}
int launch_unpermute_f64(const Launch& L, int64_t n, const double* src, const uint32_t* perm, double* dst)
{
    if (n <= 0) return 0;
    k_unpermute_f64<<<grid_n(L, n), 256, 0, L.stream>>>(n, src, perm, dst);
    return 1;
}
int launch_unpermute_f32(const Launch& L, int64_t n, const float* src, int stride, const uint32_t* perm,
                         double* dst)
{
    if (n <= 0) return 0;
    k_unpermute_f32<<<grid_n(L, n), 256, 0, L.stream>>>(n, src, stride, perm, dst);
    return 1;
}
int launch_unpermute_u32(const Launch& L, int64_t n, const uint32_t* src, const uint32_t* perm, double* dst)
{
    if (n <= 0) return 0;
    k_unpermute_u32<<<grid_n(L, n), 256, 0, L.stream>>>(n, src, perm, dst);
    return 1;
}
// inputs must be finite, with m > 0 and h > 0
__global__ void k_validate(int64_t n, State s, int* status)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const bool ok = isfinite(s.x[i]) && isfinite(s.y[i]) && isfinite(s.z[i]) && isfinite(s.vx[i]) &&
                        isfinite(s.vy[i]) && isfinite(s.vz[i]) && isfinite(s.u[i]) && s.m[i] > 0.0 &&
                        isfinite(s.m[i]) && s.h[i] > 0.0 && isfinite(s.h[i]);
        if (!ok) atomicOr(status, kStNonFinite);
    }
}

int launch_validate(const Launch& L, int64_t n, const State& s, int* status)
{
    if (n <= 0) return 0;
    k_validate<<<grid_n(L, n), 256, 0, L.stream>>>(n, s, status);
    return 1;
}

// ---------------------------------------------------------------------------
// Reused candidate supersets.  The superset built on state 0 with the search
// h g_k of every particle (g_k >= h_k0) lists every pair with
// r0 < 2 max(g_i, g_j).  It still holds every neighbour pair of the current
// state while D = max_k |x_k - x_k0| <= min_k (g_k - h_k): for a pair with
// r < 2 max(h_i, h_j), say h_i >= h_j, r0 <= r + 2 D < 2 (h_i + D) <= 2 g_i
// (distances and displacements with the minimum image along z).
// g_k = h_k (1 + skin + 3 (f_k - 1)+), f_k the factor the last step's h
// adaptation applied: particles whose h is growing (a free surface, where
// they have too few neighbours) get the room for a few more steps of it.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_skin_radius(int64_t n, State s, const uint32_t* nown, const double* hfac,
                                                     double n_target, double skin, double* hsearch)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        double f = 1.0;
        if (nown) {
            const uint32_t ni = nown[k];
            if (ni == 0) f = 2.0;
            else if (ni < (uint32_t)kHFacN) f = hfac[ni];
            else f = 0.5 * (1.0 + cbrt(n_target / (double)ni));
        }
        const double g = 1.0 + skin + 3.0 * fmax(f - 1.0, 0.0);
        hsearch[k] = s.h[k] * fmin(g, 4.0);
    }
}

int launch_skin_radius(const Launch& L, int64_t n, const State& s, const uint32_t* nown, const double* hfac,
                       double n_target, double skin, double* hsearch)
{
    if (n <= 0) return 0;
    k_skin_radius<<<grid_n(L, n), 256, 0, L.stream>>>(n, s, nown, hfac, n_target, skin, hsearch);
    return 1;
}

// positions of the build (the search h is already in ref.h0)
__global__ void __launch_bounds__(256) k_skin_snapshot(int64_t n, State s, double* x0, double* y0, double* z0)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        x0[k] = s.x[k];
        y0[k] = s.y[k];
        z0[k] = s.z[k];
    }
}

int launch_skin_snapshot(const Launch& L, int64_t n, const State& s, const SkinRef& ref)
{
    if (n <= 0) return 0;
    k_skin_snapshot<<<grid_n(L, n), 256, 0, L.stream>>>(n, s, ref.x0, ref.y0, ref.z0);
    return 1;
}

// red[0]: largest displacement, red[1]: smallest slack (ordered-integer
// encoded); both reset by k_skin_reset
__global__ void k_skin_reset(unsigned long long* red)
{
    red[0] = ord_f64(0.0);
    red[1] = ord_f64(1e300);
}

__global__ void __launch_bounds__(256) k_skin_check(int64_t n, State s, const uint16_t* patch_of, const PatchDev* pd,
                                                    SkinRef ref, unsigned long long* red)
{
    double dmax = 0.0, smin = 1e300;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const double lz = pd[patch_of[k]].lz;
        const double dx = s.x[k] - ref.x0[k], dy = s.y[k] - ref.y0[k];
        double dz = s.z[k] - ref.z0[k];
        if (dz > 0.5 * lz) dz -= lz;
        else if (dz < -0.5 * lz) dz += lz;
        dmax = fmax(dmax, sqrt(dx * dx + dy * dy + dz * dz));
        smin = fmin(smin, ref.h0[k] - s.h[k]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
        smin = fmin(smin, __shfl_xor_sync(0xffffffffu, smin, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&red[0], ord_f64(dmax));
        atomicMin(&red[1], ord_f64(smin));
    }
}

// flag = 1 while the superset holds (with a relative margin of 1e-9 against
// the rounding of the two reductions)
__global__ void k_skin_decide(const unsigned long long* red, int* flag)
{
    const double dmax = unord_f64(red[0]), smin = unord_f64(red[1]);
    *flag = (smin > 0.0 && dmax * (1.0 + 1e-9) <= smin) ? 1 : 0;
}

int launch_skin_check(const Launch& L, int64_t n, const State& s, const uint16_t* patch_of, const PatchDev* pd,
                      const SkinRef& ref, unsigned long long* red, int* flag)
{
    k_skin_reset<<<1, 1, 0, L.stream>>>(red);
    int k = 1;
    if (n > 0) {
        k_skin_check<<<grid_n(L, n), 256, 0, L.stream>>>(n, s, patch_of, pd, ref, red);
        k++;
    }
    k_skin_decide<<<1, 1, 0, L.stream>>>(red, flag);
    return k + 1;
}

}  // namespace sphg
