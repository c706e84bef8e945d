// sph_pairs.cu -- the SPH pair sums over the CSR neighbour lists (Sec. 3):
//   density  rho_i = m_i W(0, h_i) + sum_j m_j W(r_ij, h_i)        (R1, Eq. 2)
//   EOS      P = (gamma - 1) rho u,  c = sqrt(gamma P / rho)        (R9)
//   momentum a_i  = -sum_j m_j (A_i + A_j + Pi_ij) grad_i Wbar_ij   (R4)
//   energy   du_i =  sum_j m_j (A_i + Pi_ij / 2) v_ij . grad_i Wbar_ij (R6)
// with A = P / rho^2, Wbar_ij = (W(r,h_i) + W(r,h_j)) / 2 and the Monaghan
// viscosity Pi_ij = (-alpha cbar mu + beta mu^2) / rhobar for approaching
// pairs, mu = hbar v_ij . x_ij / (r^2 + eps hbar^2) (R5).
//
// Wendland kernel (Eq. 2, 1/h^3 restored): with w = 1/(2h) and
// q = 1 - r w = 1 - v/2,
//   W(r, h)         = sigma/h^3 q^4 (5 - 4 q)          (2v + 1 = 5 - 4q)
//   grad_i W(r, h)  = -160 sigma w^5 q^3 (x_i - x_j)   (5 sigma / h^5 = 160 sigma w^5)
// so grad_i Wbar_ij = -80 sigma (w_i^5 q_i^3 + w_j^5 q_j^3) (x_i - x_j), and the
// factor 80 sigma = 105/pi is applied once per particle.
//
// One group of TPP lanes per particle strides over the particle's row; the
// group reduces its partial sums with shuffles.  Mixed precision: positions
// are FP32 offsets from the particle's cell origin, the column word carries
// the stencil cell so x_i - x_j = (o_i - o_j) - dc s exactly up to FP32
// rounding of o (a neighbour beyond the 5 x 5 x 5 stencil, kFarCode, takes dc
// from both particles' cell coordinates); sums are Kahan-compensated FP32.
// FP64 path: every pair operation in double.
#include "sph_internal.cuh"

namespace sphg {


#ifndef SPH_MOM_CHUNK
#define SPH_MOM_CHUNK 1                 // momentum: row words in chunks of four (below)
#endif
#ifndef SPH_DEN_CHUNK
#define SPH_DEN_CHUNK 0                 // density: the same; measured slower there
#endif
#ifndef SPH_ROW_PREFETCH
#define SPH_ROW_PREFETCH 1              // L2 prefetch of the next particle's row
#endif

__device__ __forceinline__ void kahan_add(float& s, float& c, float v)
{
    const float y = __fsub_rn(v, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}

// Kahan step for the term a*b: the product is rounded once, inside y
__device__ __forceinline__ void kahan_fma(float& s, float& c, float a, float b)
{
    const float y = fmaf(a, b, -c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}

// merge another lane's compensated sum (value s2 - c2) into (s, c)
__device__ __forceinline__ void kahan_merge(float& s, float& c, float s2, float c2)
{
    kahan_add(s, c, s2);
    kahan_add(s, c, -c2);
}

template <int TPP>
__device__ __forceinline__ void group_kahan_reduce(float& s, float& c, unsigned gmask)
{
#pragma unroll
    for (int o = TPP / 2; o > 0; o >>= 1) {
        const float s2 = __shfl_xor_sync(gmask, s, o);
        const float c2 = __shfl_xor_sync(gmask, c, o);
        kahan_merge(s, c, s2, c2);
    }
}

template <int TPP>
__device__ __forceinline__ double group_sum(double v, unsigned gmask)
{
#pragma unroll
    for (int o = TPP / 2; o > 0; o >>= 1) v += __shfl_xor_sync(gmask, v, o);
    return v;
}

// stencil offsets of the packed column word: {dcx, dcy, dcz, t}, the z entry
// used with zmode 0, t (z cell offset, FP32 minimum image) with zmode 1
__device__ __forceinline__ void fill_stencil_table(float4* tab)
{
    for (int k = threadIdx.x; k < kStencilCells; k += blockDim.x) {
        const int zd = k / 25;
        tab[k] = make_float4((float)(k % 5 - 2), (float)((k / 5) % 5 - 2), (float)(zd - 2), (float)zd);
    }
    __syncthreads();
}

struct GroupIdx {
    int gl;
    unsigned gmask;
};

template <int TPP>
__device__ __forceinline__ GroupIdx group_idx()
{
    const int lane = threadIdx.x & 31;
    GroupIdx g;
    g.gl = lane & (TPP - 1);
    g.gmask = TPP == 32 ? 0xffffffffu : (((1u << TPP) - 1u) << (lane & ~(TPP - 1)));
    return g;
}

// pair separation x_i - x_j for a kFarCode column: the cell offset from both
// particles' cell coordinates, then the nearest image along z
__device__ __forceinline__ void rel_dx_far(uint32_t ci, uint32_t cj, float s_f, float sz_f, float lz_f, float oxi,
                                           float oyi, float ozi, const float4& q, float& dx, float& dy, float& dz)
{
    const int dcx = (int)(cj & 255u) - (int)(ci & 255u);
    const int dcy = (int)((cj >> 8) & 255u) - (int)((ci >> 8) & 255u);
    const int dcz = (int)(cj >> 16) - (int)(ci >> 16);
    dx = fmaf(-(float)dcx, s_f, oxi - q.x);
    dy = fmaf(-(float)dcy, s_f, oyi - q.y);
    dz = fmaf(-(float)dcz, sz_f, ozi - q.z);
    if (dz > 0.5f * lz_f) dz -= lz_f;
    else if (dz < -0.5f * lz_f) dz += lz_f;
}

// pair separation x_i - x_j from cell-relative FP32 coordinates; ZW = 1 when
// the patch has fewer than 2K+1 z cells (z offset as a cell count, then the
// minimum image), ZW = 0 otherwise (signed z offset, no wrap needed)
template <int ZW>
__device__ __forceinline__ void rel_dx(const float4& e, float s_f, float sz_f, float lz_f, float oxi,
                                       float oyi, float ozi, const float4& q, float& dx, float& dy, float& dz)
{
    dx = fmaf(-e.x, s_f, oxi - q.x);
    dy = fmaf(-e.y, s_f, oyi - q.y);
    dz = fmaf(-(ZW ? e.w : e.z), sz_f, ozi - q.z);
    if (ZW) {
        if (dz > 0.5f * lz_f) dz -= lz_f;
        else if (dz < -0.5f * lz_f) dz += lz_f;
    }
}

// ---------------------------------------------------------------------------
// The two kernels of Sec. 3, with w = 1/(2h):
//   Wendland (Eq. 2): W = sigma/h^3 q^4 (5 - 4q), q = 1 - r w;
//     grad_i W = -160 sigma w^5 q^3 (x_i - x_j)
//   Sinc: W = B_n/h^3 S^n, S = sin(x)/x, x = pi r w (= pi v / 2);
//     grad_i W = -8 B_n n pi^2 w^5 S^(n-1) g(x) (x_i - x_j), g = (sin x - x cos x)/x^3
// The pair loops carry only the factors that depend on r (the density
// weight, and w^5 times the shape of the gradient); the constants are
// applied once per particle: rho = 8 kb w_i^3 (sum + m_i), and grad_i Wbar
// is half the two sides' gradients, 80 sigma or 4 B_n n pi^2 times the sum
// of the two sides' factors (kb = sigma or B_n).
// ---------------------------------------------------------------------------
constexpr float kPif = 3.14159265358979323846f;
constexpr double kPi = 3.14159265358979323846;

__device__ __forceinline__ float ipowf(float b, int e)
{
    float r = 1.0f;
    for (int k = 0; k < e; k++) r *= b;
    return r;
}
__device__ __forceinline__ double ipowd(double b, int e)
{
    double r = 1.0;
    for (int k = 0; k < e; k++) r *= b;
    return r;
}

// g(x) = (sin x - x cos x)/x^3: its Taylor series sum_m (-1)^(m+1) 2m x^(2m-2)
// / (2m+1)! below x = 1, where the direct form loses digits to cancellation
__device__ __forceinline__ float sinc_g(float x, float sn, float cs)
{
    if (x < 1.0f) {
        const float x2 = x * x;
        return fmaf(x2, fmaf(x2, fmaf(x2, fmaf(x2, 1.0f / 3991680.0f, -1.0f / 45360.0f), 1.0f / 840.0f),
                             -1.0f / 30.0f),
                    1.0f / 3.0f);
    }
    return __fdividef(fmaf(-x, cs, sn), x * x * x);
}
__device__ __forceinline__ double sinc_g(double x, double sn, double cs)
{
    if (x < 1.0) {
        const double x2 = x * x;
        double t = 0.0, pw = 1.0, fact = 6.0;
        for (int m = 1; m <= 10; m++) {
            const double term = 2.0 * m * pw / fact;
            t += (m & 1) ? term : -term;
            pw *= x2;
            fact *= (2.0 * m + 2.0) * (2.0 * m + 3.0);
        }
        return t;
    }
    return (sn - x * cs) / (x * x * x);
}

template <int KERN>
struct KernF;

template <>
struct KernF<SPH_KERNEL_WENDLAND> {
    // density weight q^4 (5 - 4q)
    static __device__ __forceinline__ float dens(float r, float w, int)
    {
        const float q = fmaxf(fmaf(-r, w, 1.0f), 0.0f);
        const float q2 = q * q;
        return q2 * q2 * fmaf(-4.0f, q, 5.0f);
    }
    static __device__ __forceinline__ double dens(double r, double w, int)
    {
        const double q = fmax(1.0 - r * w, 0.0);
        const double q2 = q * q;
        return q2 * q2 * (5.0 - 4.0 * q);
    }
    // gradient factor w^5 q^3
    static __device__ __forceinline__ float grad(float r, float w, float w5, int)
    {
        const float q = fmaxf(fmaf(-r, w, 1.0f), 0.0f);
        return w5 * (q * q * q);
    }
    static __device__ __forceinline__ double grad(double r, double w, double w5, int)
    {
        const double q = fmax(1.0 - r * w, 0.0);
        return w5 * q * q * q;
    }
    static __host__ __device__ double grad_scale(double kb, int) { return 80.0 * kb; }
    // grad-h weight -v S'(v) of the shape S = q^4 (5 - 4q), q = 1 - v/2:
    // 20 (1 - q)^2 q^3, never negative, 0 at v = 0 and v >= 2
    static __device__ __forceinline__ float omega_w(float r, float w, int)
    {
        const float q = fmaxf(fmaf(-r, w, 1.0f), 0.0f);
        const float p = 1.0f - q;
        return 20.0f * (p * p) * (q * q * q);
    }
    static __device__ __forceinline__ double omega_w(double r, double w, int)
    {
        const double q = fmax(1.0 - r * w, 0.0);
        const double p = 1.0 - q;
        return 20.0 * (p * p) * (q * q * q);
    }
};

template <>
struct KernF<SPH_KERNEL_SINC> {
    static __device__ __forceinline__ float dens(float r, float w, int n)
    {
        const float x = kPif * r * w;
        if (!(x < kPif)) return 0.0f;
        float sn, cs;
        __sincosf(x, &sn, &cs);
        return ipowf(x > 0.0f ? __fdividef(sn, x) : 1.0f, n);
    }
    static __device__ __forceinline__ double dens(double r, double w, int n)
    {
        const double x = kPi * r * w;
        if (!(x < kPi)) return 0.0;
        return ipowd(x > 0.0 ? sin(x) / x : 1.0, n);
    }
    static __device__ __forceinline__ float grad(float r, float w, float w5, int n)
    {
        const float x = kPif * r * w;
        if (!(x < kPif)) return 0.0f;
        float sn, cs;
        __sincosf(x, &sn, &cs);
        const float S = x > 0.0f ? __fdividef(sn, x) : 1.0f;
        return w5 * ipowf(S, n - 1) * sinc_g(x, sn, cs);
    }
    static __device__ __forceinline__ double grad(double r, double w, double w5, int n)
    {
        const double x = kPi * r * w;
        if (!(x < kPi)) return 0.0;
        double sn, cs;
        sincos(x, &sn, &cs);
        const double S = x > 0.0 ? sn / x : 1.0;
        return w5 * ipowd(S, n - 1) * sinc_g(x, sn, cs);
    }
    static __host__ __device__ double grad_scale(double kb, int n) { return 4.0 * kb * n * kPi * kPi; }
    // grad-h weight -v d(S^n)/dv = n S^(n-1) x^2 g(x) (x = pi v / 2), never
    // negative on the support
    static __device__ __forceinline__ float omega_w(float r, float w, int n)
    {
        const float x = kPif * r * w;
        if (!(x < kPif)) return 0.0f;
        float sn, cs;
        __sincosf(x, &sn, &cs);
        const float S = x > 0.0f ? __fdividef(sn, x) : 1.0f;
        return (float)n * ipowf(S, n - 1) * (x * x) * sinc_g(x, sn, cs);
    }
    static __device__ __forceinline__ double omega_w(double r, double w, int n)
    {
        const double x = kPi * r * w;
        if (!(x < kPi)) return 0.0;
        double sn, cs;
        sincos(x, &sn, &cs);
        const double S = x > 0.0 ? sn / x : 1.0;
        return n * ipowd(S, n - 1) * (x * x) * sinc_g(x, sn, cs);
    }
};

// The list words stream from HBM (the pool is far larger than L2).  Each
// group asks L2 for the row of the particle it takes next -- the group's lanes
// cover it in 128-byte lines -- while it works on the current one; the start
// of that row was read one particle earlier, so the request does not wait.
struct RowAhead {
    unsigned long long start;
    uint32_t len;
};

__device__ __forceinline__ RowAhead row_ahead_read(const PairArgs& a, int64_t i)
{
    RowAhead r = {0ull, 0u};
    if (i < a.n) {
        r.start = a.rowstart[i];
        r.len = a.cnt[i];
    }
    return r;
}

template <int TPP>
__device__ __forceinline__ void row_ahead_prefetch(const PairArgs& a, const RowAhead& r, int gl)
{
#if SPH_ROW_PREFETCH
    for (uint32_t o = (uint32_t)gl * 32u; o < r.len; o += TPP * 32u)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(a.col + r.start + o));
#endif
}

// ---------------------------------------------------------------------------
// A5 + A6, mixed precision
// ---------------------------------------------------------------------------
// the row of one particle: plain FP32 weights m_j W-shape(r), Kahan sum
// GH: also the sum of m_j (-v S'(v)) for the grad-h factor Omega
template <int TPP, int ZW, int KERN, bool GH>
__device__ __forceinline__ void density_row(const PairArgs& a, const float4* tab, const uint32_t* row, uint32_t len,
                                            int gl, float s_f, float sz_f, float lz_f, const float4& ri, float inv2h,
                                            uint32_t ci, float& sum, float& comp, float& sumd, float& compd)
{
    const int kn = a.kernel_n;
#if SPH_DEN_CHUNK
    static_assert(!GH, "the chunked density loop has no grad-h sum");
    // chunks of four row words as in the momentum sum
    const uint4* row4 = reinterpret_cast<const uint4*>(row);
    const uint32_t nch = (len + 3u) >> 2;
    for (uint32_t ch = (uint32_t)gl; ch < nch; ch += TPP) {
        const uint4 w = row4[ch];
        const uint32_t base = ch * 4u;
        // words past the row end (inside the reservation, never written) are
        // replaced by the chunk's first word, which is in the row
        uint32_t cw[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int u = 1; u < 4; u++)
            if (base + (uint32_t)u >= len) cw[u] = w.x;
        float4 q[4];
#pragma unroll
        for (int u = 0; u < 4; u++) q[u] = a.r.r5[cw[u] & kColMask];
        float b = 0.0f;
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const uint32_t code = cw[u] >> kColBits;
            float dx, dy, dz;
            if (code != kFarCode)
                rel_dx<ZW>(tab[code], s_f, sz_f, lz_f, ri.x, ri.y, ri.z, q[u], dx, dy, dz);
            else
                rel_dx_far(ci, a.cellxyz[cw[u] & kColMask], s_f, sz_f, lz_f, ri.x, ri.y, ri.z, q[u], dx, dy, dz);
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            const float r = r2 * rsqrtf(r2 + 1e-30f);
            const float m = base + (uint32_t)u < len ? q[u].w : 0.0f;
            b = fmaf(m, KernF<KERN>::dens(r, inv2h, kn), b);
        }
        kahan_add(sum, comp, b);
    }
#else
    // four neighbours per lane and iteration: the gathers are issued together
    for (uint32_t k = gl; k < len; k += 4 * TPP) {
        uint32_t cw[4];
        float4 q[4];
#pragma unroll
        for (int u = 0; u < 4; u++) cw[u] = row[min(k + (uint32_t)(u * TPP), len - 1u)];
#pragma unroll
        for (int u = 0; u < 4; u++) q[u] = a.r.r5[cw[u] & kColMask];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const uint32_t code = cw[u] >> kColBits;
            float dx, dy, dz;
            if (code != kFarCode)
                rel_dx<ZW>(tab[code], s_f, sz_f, lz_f, ri.x, ri.y, ri.z, q[u], dx, dy, dz);
            else
                rel_dx_far(ci, a.cellxyz[cw[u] & kColMask], s_f, sz_f, lz_f, ri.x, ri.y, ri.z, q[u], dx, dy, dz);
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            const float r = r2 * rsqrtf(r2 + 1e-30f);
            const float m = k + (uint32_t)(u * TPP) < len ? q[u].w : 0.0f;
            kahan_fma(sum, comp, m, KernF<KERN>::dens(r, inv2h, kn));
            if (GH) kahan_fma(sumd, compd, m, KernF<KERN>::omega_w(r, inv2h, kn));
        }
    }
#endif
}

template <int TPP, int KERN, bool GH>
__global__ void __launch_bounds__(256) k_density_mixed(PairArgs a)
{
    const float kb8 = (float)(8.0 * a.kb);
    __shared__ float4 tab[kStencilCells];
    fill_stencil_table(tab);
    if (*a.status & kStBad) return;
    const GroupIdx G = group_idx<TPP>();
    const int64_t gs = ((int64_t)gridDim.x * blockDim.x) / TPP;
    const float gam = (float)a.gamma;
    const int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / TPP;
    RowAhead ahead = row_ahead_read(a, i0 + gs);
    for (int64_t i = i0; i < a.n; i += gs) {
        row_ahead_prefetch<TPP>(a, ahead, G.gl);
        ahead = row_ahead_read(a, i + 2 * gs);
        const PatchDev* P = a.pd + a.patch_of[i];
        const float s_f = P->s_f, sz_f = P->sz_f, lz_f = P->lz_f;
        const float4 ri = a.r.r5[i];
        const float inv2h = a.r.rv[i].w;                   // 1 / (2 h_i)
        const uint32_t* row = a.col + a.rowstart[i];
        const uint32_t len = a.cnt[i];
        const uint32_t ci = a.cellxyz[i];
        float sum = 0.0f, comp = 0.0f, sumd = 0.0f, compd = 0.0f;
        if (P->zmode)
            density_row<TPP, 1, KERN, GH>(a, tab, row, len, G.gl, s_f, sz_f, lz_f, ri, inv2h, ci, sum, comp, sumd,
                                          compd);
        else
            density_row<TPP, 0, KERN, GH>(a, tab, row, len, G.gl, s_f, sz_f, lz_f, ri, inv2h, ci, sum, comp, sumd,
                                          compd);
        group_kahan_reduce<TPP>(sum, comp, G.gmask);
        if (GH) group_kahan_reduce<TPP>(sumd, compd, G.gmask);
        if (G.gl == 0) {
            const float tot = ri.w + (sum - comp);           // self term m_i W(0) ~ m_i
            const float rho = kb8 * tot * (inv2h * inv2h * inv2h);
            const float u = a.r.uf[i];                       // specific energy, staged by the gather
            const float Pr = (gam - 1.0f) * rho * u;
            const float c = sqrtf(gam * Pr / rho);
            float A = Pr / (rho * rho);
            if (GH) {
                // R20 without cancellation: Omega = sum_j m_j (-v S'(v)) / (3 sum_j m_j S(v))
                // (the self term adds nothing above the line); A/Omega is what the
                // grad-h momentum sum uses
                const float om = (sumd - compd) / (3.0f * tot);
                A = A / om;
                if (!(om > 0.0f)) atomicOr(a.status, kStNonFinite);
            }
            const float hf = 0.5f / inv2h;
            a.r.rt[i] = make_float4(rho, A, c, hf);
            a.r.pf[i] = Pr;
            a.r.hc[i] = hf / c;
            if (!(rho > 0.0f) || !isfinite(rho) || !isfinite(Pr) || !isfinite(c))
                atomicOr(a.status, kStNonFinite);
        }
    }
}

// ---------------------------------------------------------------------------
// A5 + A6, FP64
// ---------------------------------------------------------------------------
template <int TPP, int KERN, bool GH>
__global__ void __launch_bounds__(256) k_density_fp64(PairArgs a)
{
    const int kn = a.kernel_n;
    if (*a.status & kStBad) return;
    const GroupIdx G = group_idx<TPP>();
    const int64_t gs = ((int64_t)gridDim.x * blockDim.x) / TPP;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / TPP; i < a.n; i += gs) {
        const PatchDev* P = a.pd + a.patch_of[i];
        const double lz = P->lz, hl = 0.5 * P->lz;
        const double xi = a.s.x[i], yi = a.s.y[i], zi = a.s.z[i], hi = a.s.h[i];
        const double w = 0.5 * a.f.invh[i];
        const uint32_t* row = a.col + a.rowstart[i];
        const uint32_t len = a.cnt[i];
        double sum = 0.0, sumd = 0.0;
        for (uint32_t k = G.gl; k < len; k += TPP) {
            const uint32_t j = row[k] & kColMask;
            const double dx = xi - a.s.x[j], dy = yi - a.s.y[j];
            double dz = zi - a.s.z[j];
            if (dz > hl) dz -= lz;
            else if (dz < -hl) dz += lz;
            const double r = sqrt(dx * dx + dy * dy + dz * dz);
            sum += a.s.m[j] * KernF<KERN>::dens(r, w, kn);
            if (GH) sumd += a.s.m[j] * KernF<KERN>::omega_w(r, w, kn);
        }
        sum = group_sum<TPP>(sum, G.gmask);
        if (GH) sumd = group_sum<TPP>(sumd, G.gmask);
        if (G.gl == 0) {
            const double rho = a.kb * (a.s.m[i] + sum) / (hi * hi * hi);
            const double Pr = (a.gamma - 1.0) * rho * a.s.u[i];
            const double c = sqrt(a.gamma * Pr / rho);
            a.f.rho[i] = rho;
            a.f.P[i] = Pr;
            a.f.c[i] = c;
            double A = Pr / (rho * rho);
            if (GH) {
                const double om = sumd / (3.0 * (a.s.m[i] + sum));
                A = A / om;
                if (!(om > 0.0)) atomicOr(a.status, kStNonFinite);
            }
            a.f.A[i] = A;
            a.f.hc[i] = hi / c;
            if (!(rho > 0.0) || !isfinite(rho) || !isfinite(Pr) || !isfinite(c))
                atomicOr(a.status, kStNonFinite);
        }
    }
}

// ---------------------------------------------------------------------------
// A7, mixed precision
// ---------------------------------------------------------------------------
struct PairTerms {
    float ax, ay, az, du;
};

// Per-particle constants of the momentum and energy sums.  The viscosity is
// written with sums instead of means (h_i + h_j = 2 hbar, c_i + c_j = 2 cbar,
// rho_i + rho_j = 2 rhobar), so that with m2 = (h_i + h_j) v.x / (r^2 +
// eps/4 (h_i + h_j)^2) = 2 mu,
//   Pi = mu (beta mu - alpha cbar) / rhobar
//      = m2 ((beta/2) m2 - (alpha/2)(c_i + c_j)) / (rho_i + rho_j).
struct MomConst {
    float eps4, beta2, alpha2;   // eps/4, beta/2, alpha/2
};

// one pair of the momentum and energy sums, from x_i - x_j = (dx, dy, dz);
// Wendland: w^5 q^3 = w^2 (w q)^3 with w q = w - r w^2
// GH: the grad-h form, ti.y / tj.y holding A/Omega: the pressure terms take
// each side's own kernel gradient (2 f_i, 2 f_j in units of the symmetrised one)
template <int KERN, bool GH>
__device__ __forceinline__ PairTerms momentum_pair(float dx, float dy, float dz, const float4& vi,
                                                   const float4& ti, float wi5, const float4& vj,
                                                   const float4& tj, float mj, const MomConst& K, int kn)
{
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float r = r2 * rsqrtf(r2 + 1e-30f);
    float F, fi = 0.0f, fj = 0.0f;
    if (GH) {
        const float wj2 = vj.w * vj.w;
        fi = KernF<KERN>::grad(r, vi.w, wi5, kn);
        fj = KernF<KERN>::grad(r, vj.w, wj2 * wj2 * vj.w, kn);
        F = fi + fj;
    } else if (KERN == SPH_KERNEL_WENDLAND) {
        const float qi = fmaxf(fmaf(-r, vi.w, 1.0f), 0.0f);
        const float wj2 = vj.w * vj.w;
        const float aj = fmaxf(fmaf(-r, wj2, vj.w), 0.0f);      // w_j q_j
        F = fmaf(wi5, qi * qi * qi, wj2 * (aj * aj * aj));
    } else {
        const float wj2 = vj.w * vj.w;
        F = KernF<KERN>::grad(r, vi.w, wi5, kn) + KernF<KERN>::grad(r, vj.w, wj2 * wj2 * vj.w, kn);
    }
    const float vx = vi.x - vj.x, vy = vi.y - vj.y, vz = vi.z - vj.z;
    const float vdot = fmaf(vx, dx, fmaf(vy, dy, vz * dz));
    const float hs = ti.w + tj.w;
    const float m2 = __fdividef(hs * vdot, fmaf(K.eps4 * hs, hs, r2));
    const float pi_ = vdot < 0.0f
                          ? __fdividef(m2 * fmaf(K.beta2, m2, -K.alpha2 * (ti.z + tj.z)), ti.x + tj.x)
                          : 0.0f;
    PairTerms t;
    if (GH) {
        const float pi_f = pi_ * F;
        const float fa = mj * fmaf(2.0f * ti.y, fi, fmaf(2.0f * tj.y, fj, pi_f));
        t.ax = fa * dx;
        t.ay = fa * dy;
        t.az = fa * dz;
        t.du = -mj * fmaf(2.0f * ti.y, fi, 0.5f * pi_f) * vdot;
        return t;
    }
    const float g = mj * F;
    const float fa = g * (ti.y + tj.y + pi_);
    t.ax = fa * dx;
    t.ay = fa * dy;
    t.az = fa * dz;
    t.du = -g * fmaf(0.5f, pi_, ti.y) * vdot;
    return t;
}

#ifndef SPH_MOM_PACK
#define SPH_MOM_PACK 1                  // two pairs at once in packed FP32x2 arithmetic
#endif

// packed FP32x2 helpers (one instruction for both halves)
__device__ __forceinline__ float2 p2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b, rounded once
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, p2(-1.0f), a); }

struct PairTerms2 {
    float2 ax, ay, az, du;
};

// momentum_pair for two pairs at once: the same operations, in the halves of
// packed FP32x2 values (mj = 0 in a half makes its terms 0)
__device__ __forceinline__ PairTerms2 momentum_pair2(float2 dx, float2 dy, float2 dz, const float4& vi,
                                                     const float4& ti, float wi5, const float4& va,
                                                     const float4& vb, const float4& ta, const float4& tb,
                                                     float2 mj, const MomConst& K)
{
    const float2 r2 = fma2(dx, dx, fma2(dy, dy, mul2(dz, dz)));
    const float2 r2e = add2(r2, p2(1e-30f));
    const float2 r = mul2(r2, make_float2(rsqrtf(r2e.x), rsqrtf(r2e.y)));
    const float2 qi0 = fma2(r, p2(-vi.w), p2(1.0f));
    const float2 qi = make_float2(fmaxf(qi0.x, 0.0f), fmaxf(qi0.y, 0.0f));
    const float2 wj = make_float2(va.w, vb.w);
    const float2 wj2 = mul2(wj, wj);
    const float2 aj0 = fma2(r, mul2(wj2, p2(-1.0f)), wj);
    const float2 aj = make_float2(fmaxf(aj0.x, 0.0f), fmaxf(aj0.y, 0.0f));
    const float2 F = fma2(p2(wi5), mul2(mul2(qi, qi), qi), mul2(wj2, mul2(mul2(aj, aj), aj)));
    const float2 vx = sub2(p2(vi.x), make_float2(va.x, vb.x));
    const float2 vy = sub2(p2(vi.y), make_float2(va.y, vb.y));
    const float2 vz = sub2(p2(vi.z), make_float2(va.z, vb.z));
    const float2 vdot = fma2(vx, dx, fma2(vy, dy, mul2(vz, dz)));
    const float2 hs = add2(p2(ti.w), make_float2(ta.w, tb.w));
    const float2 den = fma2(mul2(p2(K.eps4), hs), hs, r2);
    const float2 num = mul2(hs, vdot);
    const float2 m2 = mul2(num, make_float2(__fdividef(1.0f, den.x), __fdividef(1.0f, den.y)));
    const float2 cs = add2(p2(ti.z), make_float2(ta.z, tb.z));
    const float2 rs = add2(p2(ti.x), make_float2(ta.x, tb.x));
    const float2 pn = mul2(m2, fma2(p2(K.beta2), m2, mul2(p2(-K.alpha2), cs)));
    const float2 pv = mul2(pn, make_float2(__fdividef(1.0f, rs.x), __fdividef(1.0f, rs.y)));
    const float2 pi_ = make_float2(vdot.x < 0.0f ? pv.x : 0.0f, vdot.y < 0.0f ? pv.y : 0.0f);
    const float2 g = mul2(mj, F);
    const float2 fa = mul2(g, add2(add2(p2(ti.y), make_float2(ta.y, tb.y)), pi_));
    PairTerms2 t;
    t.ax = mul2(fa, dx);
    t.ay = mul2(fa, dy);
    t.az = mul2(fa, dz);
    t.du = mul2(mul2(g, p2(-1.0f)), mul2(fma2(p2(0.5f), pi_, p2(ti.y)), vdot));
    return t;
}

struct MomAcc {
    float sx, cx, sy, cy, sz, cz, su, cu;
};


// The row in chunks of four words: a lane loads its chunk with one 16-byte
// load (rows start on 32-byte boundaries and are reserved in multiples of 8
// words, so a chunk never leaves the reservation) one chunk ahead of its use,
// sums the chunk's four pair terms plainly and adds that sum with Kahan
// compensation (the plain sum of four terms errs by at most 3 eps times their
// magnitudes, the order of one term's own rounding).
template <int TPP, int ZW, int KERN, bool GH>
__device__ __forceinline__ void momentum_row(const PairArgs& a, const float4* tab, const uint32_t* row, uint32_t len,
                                             int gl, float s_f, float sz_f, float lz_f, const float4& ri,
                                             const float4& vi, const float4& ti, float wi5, const MomConst& K,
                                             uint32_t ci, MomAcc& A)
{
    const int kn = a.kernel_n;
#if SPH_MOM_CHUNK
    const uint4* row4 = reinterpret_cast<const uint4*>(row);
    const uint32_t nch = (len + 3u) >> 2;
    uint32_t ch = (uint32_t)gl;
    uint4 w = ch < nch ? row4[ch] : make_uint4(0u, 0u, 0u, 0u);
    for (; ch < nch; ch += TPP) {
        const uint4 wn = ch + TPP < nch ? row4[ch + TPP] : make_uint4(0u, 0u, 0u, 0u);
        const uint32_t cws[4] = {w.x, w.y, w.z, w.w};
        const uint32_t base = ch * 4u;
        float bx = 0.0f, by = 0.0f, bz = 0.0f, bu = 0.0f;
#if SPH_MOM_PACK
        // packed pairs: the Wendland kernel in the symmetrised form (the Sinc
        // kernel and the grad-h form take the scalar loop)
        if (KERN == SPH_KERNEL_WENDLAND && !GH) {
        float2 px = p2(0.0f), py = p2(0.0f), pz = p2(0.0f), pu = p2(0.0f);
#pragma unroll
        for (int hh = 0; hh < 2; hh++) {
            const uint32_t ua = base + 2u * hh;
            if (ua >= len) break;
            const bool hb = ua + 1u < len;
            const uint32_t cwa = cws[2 * hh], cwb = hb ? cws[2 * hh + 1] : cwa;
            const uint32_t ja = cwa & kColMask, jb = cwb & kColMask;
            const float4 qa = a.r.r5[ja], qb = a.r.r5[jb];
            const float4 va = a.r.rv[ja], vb = a.r.rv[jb];
            const float4 ta = a.r.rt[ja], tb = a.r.rt[jb];
            float dxa, dya, dza, dxb, dyb, dzb;
            const uint32_t ca = cwa >> kColBits, cb = cwb >> kColBits;
            if (ca != kFarCode) rel_dx<ZW>(tab[ca], s_f, sz_f, lz_f, ri.x, ri.y, ri.z, qa, dxa, dya, dza);
            else rel_dx_far(ci, a.cellxyz[ja], s_f, sz_f, lz_f, ri.x, ri.y, ri.z, qa, dxa, dya, dza);
            if (cb != kFarCode) rel_dx<ZW>(tab[cb], s_f, sz_f, lz_f, ri.x, ri.y, ri.z, qb, dxb, dyb, dzb);
            else rel_dx_far(ci, a.cellxyz[jb], s_f, sz_f, lz_f, ri.x, ri.y, ri.z, qb, dxb, dyb, dzb);
            const PairTerms2 t = momentum_pair2(make_float2(dxa, dxb), make_float2(dya, dyb), make_float2(dza, dzb),
                                                vi, ti, wi5, va, vb, ta, tb, make_float2(qa.w, hb ? qb.w : 0.0f), K);
            px = add2(px, t.ax);
            py = add2(py, t.ay);
            pz = add2(pz, t.az);
            pu = add2(pu, t.du);
        }
        bx = px.x + px.y;
        by = py.x + py.y;
        bz = pz.x + pz.y;
        bu = pu.x + pu.y;
        } else
#endif
#pragma unroll
        for (int u = 0; u < 4; u++) {
            if (base + (uint32_t)u >= len) break;
            const uint32_t cw = cws[u];
            const uint32_t j = cw & kColMask;
            const float4 q = a.r.r5[j];
            const float4 vj = a.r.rv[j];
            const float4 tj = a.r.rt[j];
            const uint32_t code = cw >> kColBits;
            float dx, dy, dz;
            if (code != kFarCode)
                rel_dx<ZW>(tab[code], s_f, sz_f, lz_f, ri.x, ri.y, ri.z, q, dx, dy, dz);
            else
                rel_dx_far(ci, a.cellxyz[j], s_f, sz_f, lz_f, ri.x, ri.y, ri.z, q, dx, dy, dz);
            const PairTerms t = momentum_pair<KERN, GH>(dx, dy, dz, vi, ti, wi5, vj, tj, q.w, K, kn);
            bx += t.ax;
            by += t.ay;
            bz += t.az;
            bu += t.du;
        }
        kahan_add(A.sx, A.cx, bx);
        kahan_add(A.sy, A.cy, by);
        kahan_add(A.sz, A.cz, bz);
        kahan_add(A.su, A.cu, bu);
        w = wn;
    }
#else
    for (uint32_t k = gl; k < len; k += TPP) {
        const uint32_t cw = row[k];
        const uint32_t j = cw & kColMask;
        const float4 q = a.r.r5[j];
        const float4 vj = a.r.rv[j];
        const float4 tj = a.r.rt[j];
        const uint32_t code = cw >> kColBits;
        float dx, dy, dz;
        if (code != kFarCode)
            rel_dx<ZW>(tab[code], s_f, sz_f, lz_f, ri.x, ri.y, ri.z, q, dx, dy, dz);
        else
            rel_dx_far(ci, a.cellxyz[j], s_f, sz_f, lz_f, ri.x, ri.y, ri.z, q, dx, dy, dz);
        const PairTerms t = momentum_pair<KERN, GH>(dx, dy, dz, vi, ti, wi5, vj, tj, q.w, K, kn);
        kahan_add(A.sx, A.cx, t.ax);
        kahan_add(A.sy, A.cy, t.ay);
        kahan_add(A.sz, A.cz, t.az);
        kahan_add(A.su, A.cu, t.du);
    }
#endif
}

#ifndef SPH_MOM_MINB
#define SPH_MOM_MINB 2                  // resident 256-thread CTAs per SM the registers are sized for
#endif
template <int TPP, int KERN, bool GH>
__global__ void __launch_bounds__(256, SPH_MOM_MINB) k_momentum_mixed(PairArgs a)
{
    const float gscale = (float)KernF<KERN>::grad_scale(a.kb, a.kernel_n);
    __shared__ float4 tab[kStencilCells];
    fill_stencil_table(tab);
    if (*a.status & kStBad) return;
    const GroupIdx G = group_idx<TPP>();
    const int64_t gs = ((int64_t)gridDim.x * blockDim.x) / TPP;
    const MomConst K = {0.25f * (float)a.eps, 0.5f * (float)a.beta, 0.5f * (float)a.alpha};
    const int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / TPP;
    RowAhead ahead = row_ahead_read(a, i0 + gs);
    for (int64_t i = i0; i < a.n; i += gs) {
        row_ahead_prefetch<TPP>(a, ahead, G.gl);
        ahead = row_ahead_read(a, i + 2 * gs);
        const PatchDev* P = a.pd + a.patch_of[i];
        const float s_f = P->s_f, sz_f = P->sz_f, lz_f = P->lz_f;
        const float4 ri = a.r.r5[i];
        const float4 vi = a.r.rv[i];
        const float4 ti = a.r.rt[i];
        const float wi2 = vi.w * vi.w;
        const float wi5 = wi2 * wi2 * vi.w;
        const uint32_t* row = a.col + a.rowstart[i];
        const uint32_t len = a.cnt[i];
        const uint32_t ci = a.cellxyz[i];
        MomAcc A = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (P->zmode)
            momentum_row<TPP, 1, KERN, GH>(a, tab, row, len, G.gl, s_f, sz_f, lz_f, ri, vi, ti, wi5, K, ci, A);
        else
            momentum_row<TPP, 0, KERN, GH>(a, tab, row, len, G.gl, s_f, sz_f, lz_f, ri, vi, ti, wi5, K, ci, A);
        group_kahan_reduce<TPP>(A.sx, A.cx, G.gmask);
        group_kahan_reduce<TPP>(A.sy, A.cy, G.gmask);
        group_kahan_reduce<TPP>(A.sz, A.cz, G.gmask);
        group_kahan_reduce<TPP>(A.su, A.cu, G.gmask);
        if (G.gl == 0) {
            const float4 r = make_float4(gscale * (A.sx - A.cx), gscale * (A.sy - A.cy), gscale * (A.sz - A.cz),
                                         gscale * (A.su - A.cu));
            a.r.acc[i] = r;
            if (!isfinite(r.x) || !isfinite(r.y) || !isfinite(r.z) || !isfinite(r.w))
                atomicOr(a.status, kStNonFinite);
        }
    }
}

// ---------------------------------------------------------------------------
// A7, FP64
// ---------------------------------------------------------------------------
template <int TPP, int KERN, bool GH>
__global__ void __launch_bounds__(256) k_momentum_fp64(PairArgs a)
{
    if (*a.status & kStBad) return;
    const GroupIdx G = group_idx<TPP>();
    const int64_t gs = ((int64_t)gridDim.x * blockDim.x) / TPP;
    const int kn = a.kernel_n;
    const double S80 = KernF<KERN>::grad_scale(a.kb, kn);
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / TPP; i < a.n; i += gs) {
        const PatchDev* P = a.pd + a.patch_of[i];
        const double lz = P->lz, hl = 0.5 * P->lz;
        const double xi = a.s.x[i], yi = a.s.y[i], zi = a.s.z[i];
        const double vxi = a.f.vhx[i], vyi = a.f.vhy[i], vzi = a.f.vhz[i];
        const double hi = a.s.h[i], wi = 0.5 * a.f.invh[i];
        const double wi5 = wi * wi * wi * wi * wi;
        const double rhoi = a.f.rho[i], Ai = a.f.A[i], ci = a.f.c[i];
        const uint32_t* row = a.col + a.rowstart[i];
        const uint32_t len = a.cnt[i];
        double ax = 0.0, ay = 0.0, az = 0.0, du = 0.0;
        for (uint32_t k = G.gl; k < len; k += TPP) {
            const uint32_t j = row[k] & kColMask;
            const double dx = xi - a.s.x[j], dy = yi - a.s.y[j];
            double dz = zi - a.s.z[j];
            if (dz > hl) dz -= lz;
            else if (dz < -hl) dz += lz;
            const double r2 = dx * dx + dy * dy + dz * dz;
            const double r = sqrt(r2);
            const double wj = 0.5 * a.f.invh[j];
            const double fi = KernF<KERN>::grad(r, wi, wi5, kn), fj = KernF<KERN>::grad(r, wj, wj * wj * wj * wj * wj, kn);
            const double F = fi + fj;
            const double vx = vxi - a.f.vhx[j], vy = vyi - a.f.vhy[j], vz = vzi - a.f.vhz[j];
            const double vdot = vx * dx + vy * dy + vz * dz;
            double pi_ = 0.0;
            if (vdot < 0.0) {
                const double hbar = 0.5 * (hi + a.s.h[j]);
                const double mu = hbar * vdot / (r2 + a.eps * hbar * hbar);
                pi_ = (-a.alpha * 0.5 * (ci + a.f.c[j]) * mu + a.beta * mu * mu) /
                      (0.5 * (rhoi + a.f.rho[j]));
            }
            if (GH) {
                // R20: A holds A/Omega; each side's pressure term with its own kernel
                const double fa = a.s.m[j] * (2.0 * Ai * fi + 2.0 * a.f.A[j] * fj + pi_ * F);
                ax += fa * dx;
                ay += fa * dy;
                az += fa * dz;
                du -= a.s.m[j] * (2.0 * Ai * fi + 0.5 * pi_ * F) * vdot;
            } else {
                const double g = a.s.m[j] * F;
                const double fa = g * (Ai + a.f.A[j] + pi_);
                ax += fa * dx;
                ay += fa * dy;
                az += fa * dz;
                du -= g * (Ai + 0.5 * pi_) * vdot;
            }
        }
        ax = group_sum<TPP>(ax, G.gmask);
        ay = group_sum<TPP>(ay, G.gmask);
        az = group_sum<TPP>(az, G.gmask);
        du = group_sum<TPP>(du, G.gmask);
        if (G.gl == 0) {
            a.f.ax[i] = S80 * ax;
            a.f.ay[i] = S80 * ay;
            a.f.az[i] = S80 * az;
            a.f.du[i] = S80 * du;
            if (!isfinite(ax) || !isfinite(ay) || !isfinite(az) || !isfinite(du))
                atomicOr(a.status, kStNonFinite);
        }
    }
}

#define SPH_DISPATCH_TPP(KERNEL, KERN, GH, tpp, blocks, L, a)                                   \
    switch (tpp) {                                                                              \
    case 1: KERNEL<1, KERN, GH><<<(unsigned)(blocks), 256, 0, (L).stream>>>(a); break;          \
    case 2: KERNEL<2, KERN, GH><<<(unsigned)(blocks), 256, 0, (L).stream>>>(a); break;          \
    case 4: KERNEL<4, KERN, GH><<<(unsigned)(blocks), 256, 0, (L).stream>>>(a); break;          \
    case 16: KERNEL<16, KERN, GH><<<(unsigned)(blocks), 256, 0, (L).stream>>>(a); break;        \
    case 32: KERNEL<32, KERN, GH><<<(unsigned)(blocks), 256, 0, (L).stream>>>(a); break;        \
    default: KERNEL<8, KERN, GH><<<(unsigned)(blocks), 256, 0, (L).stream>>>(a); break;         \
    }
#define SPH_DISPATCH_GH(KERNEL, KERN, tpp, blocks, L, a)                                        \
    if ((a).grad_h) {                                                                           \
        SPH_DISPATCH_TPP(KERNEL, KERN, true, tpp, blocks, L, a);                                \
    } else {                                                                                    \
        SPH_DISPATCH_TPP(KERNEL, KERN, false, tpp, blocks, L, a);                               \
    }
#define SPH_DISPATCH(KERNEL, tpp, blocks, L, a)                                                 \
    if ((a).kernel == SPH_KERNEL_SINC) {                                                        \
        SPH_DISPATCH_GH(KERNEL, SPH_KERNEL_SINC, tpp, blocks, L, a);                            \
    } else {                                                                                    \
        SPH_DISPATCH_GH(KERNEL, SPH_KERNEL_WENDLAND, tpp, blocks, L, a);                        \
    }

static int64_t pair_blocks(const Launch& L, int64_t n, int tpp)
{
    int64_t blocks = (n * tpp + 255) / 256;
    const int64_t cap = (int64_t)L.sms * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    return blocks;
}

int launch_density(const Launch& L, const PairArgs& a, int tpp, int mixed)
{
    if (a.n <= 0) return 0;
    const int64_t blocks = pair_blocks(L, a.n, tpp);
    if (mixed) {
        SPH_DISPATCH(k_density_mixed, tpp, blocks, L, a);
    } else {
        SPH_DISPATCH(k_density_fp64, tpp, blocks, L, a);
    }
    return 1;
}

int launch_momentum(const Launch& L, const PairArgs& a, int tpp, int mixed)
{
    if (a.n <= 0) return 0;
    const int64_t blocks = pair_blocks(L, a.n, tpp);
    if (mixed) {
        SPH_DISPATCH(k_momentum_mixed, tpp, blocks, L, a);
    } else {
        SPH_DISPATCH(k_momentum_fp64, tpp, blocks, L, a);
    }
    return 1;
}

}  // namespace sphg
