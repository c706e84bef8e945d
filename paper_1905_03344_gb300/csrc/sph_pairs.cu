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
#include "sph_pairmath.cuh"

namespace sphg {


#ifndef SPH_ROW_PREFETCH
#define SPH_ROW_PREFETCH 1              // L2 prefetch of the next particle's row
#endif

// The list words stream from HBM (the pool is far larger than L2) and are
// read with the streaming hint (evict first), which leaves L2 to the
// neighbour records every row gathers.  Each
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

// the positions [kb, ke) a launch covers: every particle, or a range of
// row-length bins of the order
__device__ __forceinline__ void pair_range(const PairArgs& a, int64_t& kb, int64_t& ke)
{
    if (a.order) {
        kb = a.bounds[a.bin_lo];
        ke = a.bounds[a.bin_hi + 1];
    } else {
        kb = 0;
        ke = a.n;
    }
}

// the particle at position k (a.n past the range: no particle)
__device__ __forceinline__ int64_t pair_at(const PairArgs& a, int64_t k, int64_t ke)
{
    if (k >= ke) return a.n;
    return a.order ? (int64_t)a.order[k] : k;
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
// density + EOS, mixed precision
// ---------------------------------------------------------------------------
// the row of one particle: plain FP32 weights m_j W-shape(r), Kahan sum.  A
// lane takes the row in chunks of four words (one 16-byte load; rows start on
// 32-byte boundaries and are reserved in multiples of 8 words, so a chunk
// never leaves the reservation), loaded one chunk ahead of its use, and
// issues the chunk's four record gathers together.  Words past the row end
// in the last chunk are not used as indices.
template <int TPP, int ZW, int KERN, bool GH>
__device__ __forceinline__ void density_row(const PairArgs& a, const uint32_t* row, uint32_t len,
                                            int gl, const PairSide& I, float inv2h, float& sum, float& comp,
                                            float& sumd, float& compd)
{
    const int kn = a.kernel_n;
    const PairSrc src = pair_src(a);
    const uint4* row4 = reinterpret_cast<const uint4*>(row);
    const uint32_t nch = (len + 3u) >> 2;
    uint32_t ch = (uint32_t)gl;
    uint4 w = ch < nch ? __ldcs(row4 + ch) : make_uint4(0u, 0u, 0u, 0u);
    for (; ch < nch; ch += TPP) {
        const uint4 wn = ch + TPP < nch ? __ldcs(row4 + ch + TPP) : make_uint4(0u, 0u, 0u, 0u);
        const uint32_t nv = min(len - ch * 4u, 4u);
        const uint32_t cw[4] = {w.x, nv > 1u ? w.y : w.x, nv > 2u ? w.z : w.x, nv > 3u ? w.w : w.x};
        float4 q[4];
#pragma unroll
        for (int u = 0; u < 4; u++) q[u] = src.r5[cw[u] & kColMask];
        float dx[4], dy[4], dz[4];
        // all four words within the stencil (all but the few pairs with a big
        // particle): the stencil offsets without the per-pair branch
        if (((cw[0] >> kColBits) != kFarCode) & ((cw[1] >> kColBits) != kFarCode) &
            ((cw[2] >> kColBits) != kFarCode) & ((cw[3] >> kColBits) != kFarCode)) {
#pragma unroll
            for (int u = 0; u < 4; u++)
                rel_dx<ZW>(stencil_offset(cw[u] >> kColBits), I.s_f, I.sz_f, I.lz_f, I.ncz_f, I.ri.x, I.ri.y, I.ri.z, q[u], dx[u],
                           dy[u], dz[u]);
        } else {
#pragma unroll
            for (int u = 0; u < 4; u++) col_dx<ZW>(src, I, cw[u], q[u], dx[u], dy[u], dz[u]);
        }
#pragma unroll
        for (int u = 0; u < 4; u++)
            if ((uint32_t)u < nv) density_term<KERN, GH>(dx[u], dy[u], dz[u], inv2h, kn, q[u].w, sum, comp, sumd, compd);
        w = wn;
    }
}

#ifndef SPH_DEN_MINB
#define SPH_DEN_MINB 4                  // resident 256-thread CTAs per SM the registers are sized for
#endif
template <int TPP, int KERN, bool GH>
__global__ void __launch_bounds__(256, SPH_DEN_MINB) k_density_mixed(PairArgs a)
{
    const float kb8 = (float)(8.0 * a.kb);
    if (*a.status & kStBad) return;
    const GroupIdx G = group_idx<TPP>();
    const int64_t gs = ((int64_t)gridDim.x * blockDim.x) / TPP;
    const float gam = (float)a.gamma;
    int64_t kb, ke;
    pair_range(a, kb, ke);
    const int64_t k0 = kb + ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / TPP;
    RowAhead ahead = row_ahead_read(a, pair_at(a, k0 + gs, ke));
    for (int64_t k = k0; k < ke; k += gs) {
        const int64_t i = pair_at(a, k, ke);
        row_ahead_prefetch<TPP>(a, ahead, G.gl);
        ahead = row_ahead_read(a, pair_at(a, k + 2 * gs, ke));
        const PatchDev* P = a.pd + a.patch_of[i];
        const PairSide I = pair_side(a, P, i);
        const float inv2h = a.r.rv[i].w;                   // 1 / (2 h_i)
        const uint32_t* row = a.col + a.rowstart[i];
        const uint32_t len = a.cnt[i];
        float sum = 0.0f, comp = 0.0f, sumd = 0.0f, compd = 0.0f;
        if (P->zmode) density_row<TPP, 1, KERN, GH>(a, row, len, G.gl, I, inv2h, sum, comp, sumd, compd);
        else density_row<TPP, 0, KERN, GH>(a, row, len, G.gl, I, inv2h, sum, comp, sumd, compd);
        group_kahan_reduce<TPP>(sum, comp, G.gmask);
        if (GH) group_kahan_reduce<TPP>(sumd, compd, G.gmask);
        if (G.gl == 0) density_finish<GH>(a, i, I.ri.w, inv2h, kb8, gam, sum, comp, sumd, compd);
    }
}

// ---------------------------------------------------------------------------
// density + EOS, FP64
// ---------------------------------------------------------------------------
template <int TPP, int KERN, bool GH>
__global__ void __launch_bounds__(256) k_density_fp64(PairArgs a)
{
    const int kn = a.kernel_n;
    if (*a.status & kStBad) return;
    const GroupIdx G = group_idx<TPP>();
    const int64_t gs = ((int64_t)gridDim.x * blockDim.x) / TPP;
    int64_t kb, ke;
    pair_range(a, kb, ke);
    for (int64_t k = kb + ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / TPP; k < ke; k += gs) {
        const int64_t i = pair_at(a, k, ke);
        const PatchDev* P = a.pd + a.patch_of[i];
        const double xi = a.s.x[i], yi = a.s.y[i], zi = a.s.z[i];
        const double w = a.f.w[i];
        const uint32_t* row = a.col + a.rowstart[i];
        const uint32_t len = a.cnt[i];
        double sum = 0.0, sumd = 0.0;
        for (uint32_t k = G.gl; k < len; k += TPP)
            density_pair_fp64<KERN, GH>(a, xi, yi, zi, w, P->lz, kn, __ldcs(row + k) & kColMask, sum, sumd);
        sum = group_sum<TPP>(sum, G.gmask);
        if (GH) sumd = group_sum<TPP>(sumd, G.gmask);
        if (G.gl == 0) density_finish_fp64<GH>(a, i, sum, sumd);
    }
}

// ---------------------------------------------------------------------------
// momentum + energy, mixed precision
// ---------------------------------------------------------------------------
// The row in chunks of four words: a lane loads its chunk with one 16-byte
// load (rows start on 32-byte boundaries and are reserved in multiples of 8
// words, so a chunk never leaves the reservation) one chunk ahead of its use,
// sums the chunk's four pair terms plainly and adds that sum with Kahan
// compensation (the plain sum of four terms errs by at most 3 eps times their
// magnitudes, the order of one term's own rounding).
template <int TPP, int ZW, int KERN, bool GH>
__device__ __forceinline__ void momentum_row(const PairArgs& a, const uint32_t* row, uint32_t len,
                                             int gl, const PairSide& I, const float4& vi, const float4& ti, float wi5,
                                             const MomConst& K, MomAcc& A)
{
    const int kn = a.kernel_n;
    const PairSrc src = pair_src(a);
    const uint4* row4 = reinterpret_cast<const uint4*>(row);
    const uint32_t nch = (len + 3u) >> 2;
    uint32_t ch = (uint32_t)gl;
    uint4 w = ch < nch ? __ldcs(row4 + ch) : make_uint4(0u, 0u, 0u, 0u);
    for (; ch < nch; ch += TPP) {
        const uint4 wn = ch + TPP < nch ? __ldcs(row4 + ch + TPP) : make_uint4(0u, 0u, 0u, 0u);
        const uint32_t cws[4] = {w.x, w.y, w.z, w.w};
        const uint32_t nv = min(len - ch * 4u, 4u);
        float bx, by, bz, bu;
        momentum_chunk<ZW, KERN, GH>(src, I, vi, ti, wi5, K, kn, cws, nv, bx, by, bz, bu, GlobalRecs{src});
        mom_acc_add(A, bx, by, bz, bu);
        w = wn;
    }
}

#ifndef SPH_MOM_MINB
#define SPH_MOM_MINB 2                  // resident 256-thread CTAs per SM the registers are sized for
#endif
template <int TPP, int KERN, bool GH>
__global__ void __launch_bounds__(256, SPH_MOM_MINB) k_momentum_mixed(PairArgs a)
{
    const float gscale = (float)KernF<KERN>::grad_scale(a.kb, a.kernel_n);
    if (*a.status & kStBad) return;
    const GroupIdx G = group_idx<TPP>();
    const int64_t gs = ((int64_t)gridDim.x * blockDim.x) / TPP;
    const MomConst K = {0.25f * (float)a.eps, 0.5f * (float)a.beta, 0.5f * (float)a.alpha};
    int64_t kb, ke;
    pair_range(a, kb, ke);
    const int64_t k0 = kb + ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / TPP;
    RowAhead ahead = row_ahead_read(a, pair_at(a, k0 + gs, ke));
    for (int64_t k = k0; k < ke; k += gs) {
        const int64_t i = pair_at(a, k, ke);
        row_ahead_prefetch<TPP>(a, ahead, G.gl);
        ahead = row_ahead_read(a, pair_at(a, k + 2 * gs, ke));
        const PatchDev* P = a.pd + a.patch_of[i];
        const PairSide I = pair_side(a, P, i);
        const float4 vi = a.r.rv[i];
        const float4 ti = a.r.rt[i];
        const float wi2 = vi.w * vi.w;
        const float wi5 = wi2 * wi2 * vi.w;
        const uint32_t* row = a.col + a.rowstart[i];
        const uint32_t len = a.cnt[i];
        MomAcc A = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (P->zmode) momentum_row<TPP, 1, KERN, GH>(a, row, len, G.gl, I, vi, ti, wi5, K, A);
        else momentum_row<TPP, 0, KERN, GH>(a, row, len, G.gl, I, vi, ti, wi5, K, A);
        group_kahan_reduce<TPP>(A.sx, A.cx, G.gmask);
        group_kahan_reduce<TPP>(A.sy, A.cy, G.gmask);
        group_kahan_reduce<TPP>(A.sz, A.cz, G.gmask);
        group_kahan_reduce<TPP>(A.su, A.cu, G.gmask);
        if (G.gl == 0) momentum_finish(a, i, gscale, A);
    }
}

// ---------------------------------------------------------------------------
// momentum + energy, FP64
// ---------------------------------------------------------------------------
template <int TPP, int KERN, bool GH>
__global__ void __launch_bounds__(256) k_momentum_fp64(PairArgs a)
{
    if (*a.status & kStBad) return;
    const GroupIdx G = group_idx<TPP>();
    const int64_t gs = ((int64_t)gridDim.x * blockDim.x) / TPP;
    const int kn = a.kernel_n;
    const double S80 = KernF<KERN>::grad_scale(a.kb, kn);
    int64_t kb, ke;
    pair_range(a, kb, ke);
    for (int64_t k = kb + ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / TPP; k < ke; k += gs) {
        const int64_t i = pair_at(a, k, ke);
        const PatchDev* P = a.pd + a.patch_of[i];
        const SideD I = side_fp64(a, P, i);
        const uint32_t* row = a.col + a.rowstart[i];
        const uint32_t len = a.cnt[i];
        double ax = 0.0, ay = 0.0, az = 0.0, du = 0.0;
        for (uint32_t k = G.gl; k < len; k += TPP) {
            const PairTermsD t = momentum_pair_fp64<KERN, GH>(a, I, __ldcs(row + k) & kColMask, kn);
            ax += t.ax;
            ay += t.ay;
            az += t.az;
            du += t.du;
        }
        ax = group_sum<TPP>(ax, G.gmask);
        ay = group_sum<TPP>(ay, G.gmask);
        az = group_sum<TPP>(az, G.gmask);
        du = group_sum<TPP>(du, G.gmask);
        if (G.gl == 0) momentum_finish_fp64(a, i, S80, ax, ay, az, du);
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

// One launch per run of octaves that share a lanes-per-particle value (the
// bin sizes stay on the device, so every launch takes the full grid and
// strides over its range; a launch whose range is empty returns at once).
template <class F>
static int binned_launches(PairArgs a, int w, F&& launch_one)
{
    if (a.n <= 0 || !a.order) return 0;
    int launches = 0;
    int o = 0;
    while (o < kPairOctaves) {
        const int t = octave_tpp(o, w);
        int e = o;
        while (e + 1 < kPairOctaves && octave_tpp(e + 1, w) == t) e++;
        a.bin_lo = o;
        a.bin_hi = e;
        launches += launch_one(a, t);
        o = e + 1;
    }
    return launches;
}

int launch_density_binned(const Launch& L, PairArgs a, int w, int mixed)
{
    return binned_launches(a, w, [&](const PairArgs& b, int t) { return launch_density(L, b, t, mixed); });
}

int launch_momentum_binned(const Launch& L, PairArgs a, int w, int mixed)
{
    return binned_launches(a, w, [&](const PairArgs& b, int t) { return launch_momentum(L, b, t, mixed); });
}

}  // namespace sphg
