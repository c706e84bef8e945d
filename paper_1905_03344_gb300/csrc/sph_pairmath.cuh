// sph_pairmath.cuh -- the arithmetic of one pair of the SPH sums (Sec. 3),
// shared by the sums over the neighbour lists (sph_pairs.cu) and the
// list-free sums (sph_fused.cu): compensated FP32 accumulation, the pair
// separation from cell-relative FP32 coordinates, the two kernels of Sec. 3
// and one pair of the momentum and energy sums.
#pragma once
#include "sph_internal.cuh"

namespace sphg {

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

// the stencil offsets of a column word's code (< 125): {dcx, dcy, dcz, zd},
// dcz used with zmode 0, zd (the z cell count, FP32 minimum image) with zmode
// 1.  Integer arithmetic instead of a table (no shared-memory load per pair):
// zd = code / 25 as (code 1311) >> 15 and r / 5 as (r 13) >> 6, both exact
// for code < 125, and each small integer n converted as the float 2^23 + n,
// whose bits are 0x4B000000 | n, minus 2^23 (exact)
__device__ __forceinline__ float4 stencil_offset(uint32_t code)
{
    const uint32_t zd = (code * 1311u) >> 15;
    const uint32_t r = code - 25u * zd;
    const uint32_t yd = (r * 13u) >> 6;
    const uint32_t xd = r - 5u * yd;
    const float fz = __uint_as_float(0x4B000000u | zd);
    return make_float4(__uint_as_float(0x4B000000u | xd) - 8388610.0f, __uint_as_float(0x4B000000u | yd) - 8388610.0f,
                       fz - 8388610.0f, fz - 8388608.0f);
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
// the patch has fewer than 2K+1 z cells (z offset as a cell count modulo the
// ncz cells of the period, then the minimum image), ZW = 0 otherwise (signed z
// offset, no wrap needed).  With ZW the cell count is first taken to its
// representative in [-ncz/2, ncz/2] (the half-period tie by the sign of the
// offset difference), so that (j, i) takes exactly the negated shift of
// (i, j): every step below is then symmetric under negation and the two
// separations are exact negatives, as they are without ZW.
template <int ZW>
__device__ __forceinline__ void rel_dx(const float4& e, float s_f, float sz_f, float lz_f, float ncz_f, float oxi,
                                       float oyi, float ozi, const float4& q, float& dx, float& dy, float& dz)
{
    dx = fmaf(-e.x, s_f, oxi - q.x);
    dy = fmaf(-e.y, s_f, oyi - q.y);
    const float d = ozi - q.z;
    float k = ZW ? e.w : e.z;
    if (ZW && (2.0f * k > ncz_f || (2.0f * k == ncz_f && d < 0.0f))) k -= ncz_f;
    dz = fmaf(-k, sz_f, d);
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
    return fma(-x, cs, sn) / (x * x * x);
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
        const double q = fmax(fma(-r, w, 1.0), 0.0);
        const double q2 = q * q;
        return q2 * q2 * fma(-4.0, q, 5.0);
    }
    // gradient factor w^5 q^3
    static __device__ __forceinline__ float grad(float r, float w, float w5, int)
    {
        const float q = fmaxf(fmaf(-r, w, 1.0f), 0.0f);
        return w5 * (q * q * q);
    }
    static __device__ __forceinline__ double grad(double r, double w, double w5, int)
    {
        const double q = fmax(fma(-r, w, 1.0), 0.0);
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
        const double q = fmax(fma(-r, w, 1.0), 0.0);
        const double p = 1.0 - q;
        return 20.0 * (p * p) * (q * q * q);
    }
    // dens and omega_w from one evaluation of q
    template <typename T>
    static __device__ __forceinline__ void dens_omega(T r, T w, int n, T& d, T& g)
    {
        d = dens(r, w, n);
        g = omega_w(r, w, n);
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
    // dens and omega_w from one sin/cos and one power S^(n-1)
    static __device__ __forceinline__ void dens_omega(float r, float w, int n, float& d, float& g)
    {
        const float x = kPif * r * w;
        if (!(x < kPif)) {
            d = g = 0.0f;
            return;
        }
        float sn, cs;
        __sincosf(x, &sn, &cs);
        const float S = x > 0.0f ? __fdividef(sn, x) : 1.0f;
        const float Sn1 = ipowf(S, n - 1);
        d = Sn1 * S;
        g = (float)n * Sn1 * (x * x) * sinc_g(x, sn, cs);
    }
    static __device__ __forceinline__ void dens_omega(double r, double w, int n, double& d, double& g)
    {
        const double x = kPi * r * w;
        if (!(x < kPi)) {
            d = g = 0.0;
            return;
        }
        double sn, cs;
        sincos(x, &sn, &cs);
        const double S = x > 0.0 ? sn / x : 1.0;
        const double Sn1 = ipowd(S, n - 1);
        d = Sn1 * S;
        g = n * Sn1 * (x * x) * sinc_g(x, sn, cs);
    }
};

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
    // F is the sum of the two sides' factors, each evaluated in the same form
    // and added without contraction, so that it has the same bits for
    // (i, j) and (j, i): the pair's force terms on i and on j are then exact
    // negatives (for equal masses), and the sums conserve momentum to the
    // rounding of the row sums alone
    if (GH) {
        const float wj2 = vj.w * vj.w;
        fi = KernF<KERN>::grad(r, vi.w, wi5, kn);
        fj = KernF<KERN>::grad(r, vj.w, wj2 * wj2 * vj.w, kn);
        F = __fadd_rn(fi, fj);
    } else if (KERN == SPH_KERNEL_WENDLAND) {
        const float wi2 = vi.w * vi.w, wj2 = vj.w * vj.w;
        const float ai = fmaxf(fmaf(-r, wi2, vi.w), 0.0f);      // w_i q_i
        const float aj = fmaxf(fmaf(-r, wj2, vj.w), 0.0f);      // w_j q_j
        F = __fadd_rn(__fmul_rn(wi2, ai * ai * ai), __fmul_rn(wj2, aj * aj * aj));
    } else {
        const float wj2 = vj.w * vj.w;
        F = __fadd_rn(KernF<KERN>::grad(r, vi.w, wi5, kn), KernF<KERN>::grad(r, vj.w, wj2 * wj2 * vj.w, kn));
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
        // (2 A_i f_i + 2 A_j f_j) + Pi F: symmetric in i and j, as F is
        const float fa = mj * __fadd_rn(__fadd_rn(__fmul_rn(2.0f * ti.y, fi), __fmul_rn(2.0f * tj.y, fj)), pi_f);
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

struct MomAcc {
    float sx, cx, sy, cy, sz, cz, su, cu;
};

__device__ __forceinline__ void mom_acc_add(MomAcc& A, float bx, float by, float bz, float bu)
{
    kahan_add(A.sx, A.cx, bx);
    kahan_add(A.sy, A.cy, by);
    kahan_add(A.sz, A.cz, bz);
    kahan_add(A.su, A.cu, bu);
}

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

// momentum_pair (Wendland, symmetrised form) for two pairs at once: the same
// operations, in the halves of packed FP32x2 values (mj = 0 in a half makes
// its terms 0)
__device__ __forceinline__ PairTerms2 momentum_pair2(float2 dx, float2 dy, float2 dz, const float4& vi,
                                                     const float4& ti, const float4& va,
                                                     const float4& vb, const float4& ta, const float4& tb,
                                                     float2 mj, const MomConst& K)
{
    const float2 r2 = fma2(dx, dx, fma2(dy, dy, mul2(dz, dz)));
    const float2 r2e = add2(r2, p2(1e-30f));
    const float2 r = mul2(r2, make_float2(rsqrtf(r2e.x), rsqrtf(r2e.y)));
    // both sides' factors w^2 (w q)^3 in the same form (F has the same bits
    // for (i, j) and (j, i), as in momentum_pair)
    const float wi2 = vi.w * vi.w;
    const float2 ai0 = fma2(r, p2(-wi2), p2(vi.w));
    const float2 ai = make_float2(fmaxf(ai0.x, 0.0f), fmaxf(ai0.y, 0.0f));
    const float2 wj = make_float2(va.w, vb.w);
    const float2 wj2 = mul2(wj, wj);
    const float2 aj0 = fma2(r, mul2(wj2, p2(-1.0f)), wj);
    const float2 aj = make_float2(fmaxf(aj0.x, 0.0f), fmaxf(aj0.y, 0.0f));
    const float2 F = add2(mul2(p2(wi2), mul2(mul2(ai, ai), ai)), mul2(wj2, mul2(mul2(aj, aj), aj)));
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

// ---------------------------------------------------------------------------
// One pair (or chunk of pairs) of the mixed sums, from a column word
// j | stencil code << kColBits.  The sums over the lists and the list-free
// sums call the same functions in the same order per particle, so with one
// lane per particle both give the same bits.
// ---------------------------------------------------------------------------
// what a pair reads of particle j
struct PairSrc {
    const float4* r5;          // {ox, oy, oz, m}
    const float4* rv;          // {vx, vy, vz, 1/(2h)}
    const float4* rt;          // {rho, A (or A/Omega), c, h}
    const uint32_t* cellxyz;   // cell coordinates, for kFarCode columns
};

__device__ __forceinline__ PairSrc pair_src(const PairArgs& a) { return PairSrc{a.r.r5, a.r.rv, a.r.rt, a.cellxyz}; }

// particle i's position and cell geometry
struct PairSide {
    float4 ri;                 // r5 of i
    uint32_t ci;               // cell of i
    float s_f, sz_f, lz_f;     // cell edges and z period of i's patch
    float ncz_f;               // z cells of the period
};

__device__ __forceinline__ PairSide pair_side(const PairArgs& a, const PatchDev* P, int64_t i)
{
    return PairSide{a.r.r5[i], a.cellxyz[i], P->s_f, P->sz_f, P->lz_f, (float)P->ncz};
}

// x_i - x_j for column word cw, q = r5 of j
template <int ZW>
__device__ __forceinline__ void col_dx(const PairSrc& src, const PairSide& I, uint32_t cw,
                                       const float4& q, float& dx, float& dy, float& dz)
{
    const uint32_t code = cw >> kColBits;
    if (code != kFarCode)
        rel_dx<ZW>(stencil_offset(code), I.s_f, I.sz_f, I.lz_f, I.ncz_f, I.ri.x, I.ri.y, I.ri.z, q, dx, dy, dz);
    else
        rel_dx_far(I.ci, src.cellxyz[cw & kColMask], I.s_f, I.sz_f, I.lz_f, I.ri.x, I.ri.y, I.ri.z, q, dx, dy, dz);
}

// density: one Kahan step of m W-shape(r) (and of m (-v S'(v)) for grad-h),
// from x_i - x_j = (dx, dy, dz)
template <int KERN, bool GH>
__device__ __forceinline__ void density_term(float dx, float dy, float dz, float inv2h, int kn, float m, float& sum,
                                             float& comp, float& sumd, float& compd)
{
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float r = r2 * rsqrtf(r2 + 1e-30f);
    if (GH) {
        float d, g;
        KernF<KERN>::dens_omega(r, inv2h, kn, d, g);
        kahan_fma(sum, comp, m, d);
        kahan_fma(sumd, compd, m, g);
    } else {
        kahan_fma(sum, comp, m, KernF<KERN>::dens(r, inv2h, kn));
    }
}

// the same for column word cw, q = r5 of j
template <int ZW, int KERN, bool GH>
__device__ __forceinline__ void density_pair(const PairSrc& src, const PairSide& I, float inv2h,
                                             int kn, uint32_t cw, const float4& q, float m, float& sum, float& comp,
                                             float& sumd, float& compd)
{
    float dx, dy, dz;
    col_dx<ZW>(src, I, cw, q, dx, dy, dz);
    density_term<KERN, GH>(dx, dy, dz, inv2h, kn, m, sum, comp, sumd, compd);
}

// density epilogue of particle i: rho from the shape sum (self term m_i),
// EOS, and the records the momentum sum reads
template <bool GH>
__device__ __forceinline__ void density_finish(const PairArgs& a, int64_t i, float mi, float inv2h, float kb8,
                                               float gam, float sum, float comp, float sumd, float compd)
{
    const float tot = mi + (sum - comp);                 // self term m_i W(0) ~ m_i
    const float rho = kb8 * tot * (inv2h * inv2h * inv2h);
    const float u = a.r.uf[i];                           // specific energy, staged by the gather
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
    if (!(rho > 0.0f) || !isfinite(rho) || !isfinite(Pr) || !isfinite(c)) atomicOr(a.status, kStNonFinite);
}

#ifndef SPH_MOM_PACK
#define SPH_MOM_PACK 1                  // two pairs at once in packed FP32x2 arithmetic
#endif

// the records of pair u of a chunk straight from the record arrays
struct GlobalRecs {
    const PairSrc& src;
    __device__ __forceinline__ void load(int, uint32_t cw, float4& q, float4& v, float4& t) const
    {
        const uint32_t j = cw & kColMask;
        q = src.r5[j];
        v = src.rv[j];
        t = src.rt[j];
    }
};

// momentum: the plain sums (bx, by, bz, bu) of up to four pairs, the column
// words cws[0 .. nv), the records of pair u from R.load(u, ...)
template <int ZW, int KERN, bool GH, class Recs4 = GlobalRecs>
__device__ __forceinline__ void momentum_chunk(const PairSrc& src, const PairSide& I,
                                               const float4& vi, const float4& ti, float wi5, const MomConst& K,
                                               int kn, const uint32_t (&cws)[4], uint32_t nv, float& bx, float& by,
                                               float& bz, float& bu, const Recs4& R)
{
    bx = by = bz = bu = 0.0f;
    // packed pairs: the Wendland kernel in the symmetrised form (the Sinc
    // kernel and the grad-h form take the scalar loop)
    if constexpr (SPH_MOM_PACK && KERN == SPH_KERNEL_WENDLAND && !GH) {
        float2 px = p2(0.0f), py = p2(0.0f), pz = p2(0.0f), pu = p2(0.0f);
#pragma unroll
        for (int hh = 0; hh < 2; hh++) {
            const uint32_t ua = 2u * hh;
            if (ua >= nv) break;
            const bool hb = ua + 1u < nv;
            const uint32_t cwa = cws[2 * hh], cwb = hb ? cws[2 * hh + 1] : cwa;
            float4 qa, qb, va, vb, ta, tb;
            R.load(2 * hh, cwa, qa, va, ta);
            R.load(hb ? 2 * hh + 1 : 2 * hh, cwb, qb, vb, tb);
            float dxa, dya, dza, dxb, dyb, dzb;
            // both words within the stencil (all but the few pairs with a big
            // particle): the stencil offsets without the per-pair branch
            if (((cwa >> kColBits) != kFarCode) & ((cwb >> kColBits) != kFarCode)) {
                rel_dx<ZW>(stencil_offset(cwa >> kColBits), I.s_f, I.sz_f, I.lz_f, I.ncz_f, I.ri.x, I.ri.y, I.ri.z, qa, dxa, dya, dza);
                rel_dx<ZW>(stencil_offset(cwb >> kColBits), I.s_f, I.sz_f, I.lz_f, I.ncz_f, I.ri.x, I.ri.y, I.ri.z, qb, dxb, dyb, dzb);
            } else {
                col_dx<ZW>(src, I, cwa, qa, dxa, dya, dza);
                col_dx<ZW>(src, I, cwb, qb, dxb, dyb, dzb);
            }
            const PairTerms2 t = momentum_pair2(make_float2(dxa, dxb), make_float2(dya, dyb), make_float2(dza, dzb),
                                                vi, ti, va, vb, ta, tb, make_float2(qa.w, hb ? qb.w : 0.0f), K);
            px = add2(px, t.ax);
            py = add2(py, t.ay);
            pz = add2(pz, t.az);
            pu = add2(pu, t.du);
        }
        bx = px.x + px.y;
        by = py.x + py.y;
        bz = pz.x + pz.y;
        bu = pu.x + pu.y;
    } else {
#pragma unroll
        for (int u = 0; u < 4; u++) {
            if ((uint32_t)u >= nv) break;
            const uint32_t cw = cws[u];
            float4 q, vj, tj;
            R.load(u, cw, q, vj, tj);
            float dx, dy, dz;
            col_dx<ZW>(src, I, cw, q, dx, dy, dz);
            const PairTerms t = momentum_pair<KERN, GH>(dx, dy, dz, vi, ti, wi5, vj, tj, q.w, K, kn);
            bx += t.ax;
            by += t.ay;
            bz += t.az;
            bu += t.du;
        }
    }
}

// momentum epilogue of particle i
__device__ __forceinline__ void momentum_finish(const PairArgs& a, int64_t i, float gscale, const MomAcc& A)
{
    const float4 r = make_float4(gscale * (A.sx - A.cx), gscale * (A.sy - A.cy), gscale * (A.sz - A.cz),
                                 gscale * (A.su - A.cu));
    a.r.acc[i] = r;
    if (!isfinite(r.x) || !isfinite(r.y) || !isfinite(r.z) || !isfinite(r.w)) atomicOr(a.status, kStNonFinite);
}

// ---------------------------------------------------------------------------
// One pair of the FP64 sums: every operation in double, every multiply-add
// written as fma (the compiler may not contract a product into a sum in one
// kernel and keep it apart in another)
// ---------------------------------------------------------------------------
// x_i - x_j with the minimum image along z
__device__ __forceinline__ void pair_dx_fp64(const State& s, double xi, double yi, double zi, uint32_t j, double lz,
                                             double& dx, double& dy, double& dz)
{
    dx = xi - s.x[j];
    dy = yi - s.y[j];
    dz = zi - s.z[j];
    if (dz > 0.5 * lz) dz -= lz;
    else if (dz < -0.5 * lz) dz += lz;
}

template <int KERN, bool GH>
__device__ __forceinline__ void density_pair_fp64(const PairArgs& a, double xi, double yi, double zi, double w,
                                                  double lz, int kn, uint32_t j, double& sum, double& sumd)
{
    double dx, dy, dz;
    pair_dx_fp64(a.s, xi, yi, zi, j, lz, dx, dy, dz);
    const double r = sqrt(fma(dx, dx, fma(dy, dy, dz * dz)));
    const double m = a.s.m[j];
    if (GH) {
        double d, g;
        KernF<KERN>::dens_omega(r, w, kn, d, g);
        sum = fma(m, d, sum);
        sumd = fma(m, g, sumd);
    } else {
        sum = fma(m, KernF<KERN>::dens(r, w, kn), sum);
    }
}

template <bool GH>
__device__ __forceinline__ void density_finish_fp64(const PairArgs& a, int64_t i, double sum, double sumd)
{
    const double hi = a.s.h[i];
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
    if (!(rho > 0.0) || !isfinite(rho) || !isfinite(Pr) || !isfinite(c)) atomicOr(a.status, kStNonFinite);
}

// particle i's values for the FP64 momentum sum
struct SideD {
    double x, y, z, vx, vy, vz, h, w, w5, rho, A, c, lz;
};

__device__ __forceinline__ SideD side_fp64(const PairArgs& a, const PatchDev* P, int64_t i)
{
    SideD I;
    I.x = a.s.x[i];
    I.y = a.s.y[i];
    I.z = a.s.z[i];
    I.vx = a.f.vhx[i];
    I.vy = a.f.vhy[i];
    I.vz = a.f.vhz[i];
    I.h = a.s.h[i];
    I.w = a.f.w[i];
    I.w5 = a.f.w5[i];
    I.rho = a.f.rho[i];
    I.A = a.f.A[i];
    I.c = a.f.c[i];
    I.lz = P->lz;
    return I;
}

struct PairTermsD {
    double ax, ay, az, du;
};

// one pair of the momentum and energy sums (R4-R6; R20 with GH, A holding A/Omega)
template <int KERN, bool GH>
__device__ __forceinline__ PairTermsD momentum_pair_fp64(const PairArgs& a, const SideD& I, uint32_t j, int kn)
{
    double dx, dy, dz;
    pair_dx_fp64(a.s, I.x, I.y, I.z, j, I.lz, dx, dy, dz);
    const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
    const double r = sqrt(r2);
    const double fi = KernF<KERN>::grad(r, I.w, I.w5, kn), fj = KernF<KERN>::grad(r, a.f.w[j], a.f.w5[j], kn);
    const double F = __dadd_rn(fi, fj);   // not contracted with either product
    const double vx = I.vx - a.f.vhx[j], vy = I.vy - a.f.vhy[j], vz = I.vz - a.f.vhz[j];
    const double vdot = fma(vx, dx, fma(vy, dy, vz * dz));
    double pi_ = 0.0;
    if (vdot < 0.0) {
        // Pi = mu (beta mu - alpha cbar) / rhobar with mu = N / D, N = hbar v.x,
        // D = r^2 + eps hbar^2, as one division: N (beta N - alpha cbar D) / (D^2 rhobar)
        const double hbar = 0.5 * (I.h + a.s.h[j]);
        const double N = hbar * vdot, D = fma(a.eps * hbar, hbar, r2);
        const double cbar = 0.5 * (I.c + a.f.c[j]), rhobar = 0.5 * (I.rho + a.f.rho[j]);
        pi_ = N * fma(a.beta, N, -a.alpha * cbar * D) / (D * D * rhobar);
    }
    const double mj = a.s.m[j];
    PairTermsD t;
    if (GH) {
        // each side's pressure term with its own kernel
        const double fa = mj * fma(2.0 * I.A, fi, fma(2.0 * a.f.A[j], fj, pi_ * F));
        t.ax = fa * dx;
        t.ay = fa * dy;
        t.az = fa * dz;
        t.du = -mj * fma(2.0 * I.A, fi, 0.5 * pi_ * F) * vdot;
    } else {
        const double g = mj * F;
        const double fa = g * (I.A + a.f.A[j] + pi_);
        t.ax = fa * dx;
        t.ay = fa * dy;
        t.az = fa * dz;
        t.du = -g * fma(0.5, pi_, I.A) * vdot;
    }
    return t;
}

__device__ __forceinline__ void momentum_finish_fp64(const PairArgs& a, int64_t i, double S, double ax, double ay,
                                                     double az, double du)
{
    a.f.ax[i] = S * ax;
    a.f.ay[i] = S * ay;
    a.f.az[i] = S * az;
    a.f.du[i] = S * du;
    if (!isfinite(ax) || !isfinite(ay) || !isfinite(az) || !isfinite(du)) atomicOr(a.status, kStNonFinite);
}

}  // namespace sphg
