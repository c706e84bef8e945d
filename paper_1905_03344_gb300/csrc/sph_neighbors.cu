// sph_neighbors.cu -- neighbour discovery, second half: symmetric neighbour
// lists (Table 1 "Neighbour Discovery", symmetric union reading R11): j is
// in N(i) iff j != i and r_ij^2 < 4 h_i^2 or r_ij^2 < 4 h_j^2, with the
// minimum image along periodic z.  n_i = #{j : r_ij^2 < 4 h_i^2} feeds the
// smoothing-length adaptation.
//
// One warp serves 32 consecutive sorted particles of one patch, one lane per
// particle.  The warp expresses its particles in the frame of a reference
// cell, takes their bounding box, and enumerates the block of cells around
// it, keeping the non-empty cells closer than 2 max(h_warp, h_max(cell)).
// The candidates of the kept cells are staged 32 at a time in shared memory
// (shifted into the reference frame) and every lane tests all 32 against its
// own particle, so each candidate is loaded once per warp and the inner loop
// is a shared-memory broadcast plus FP32 arithmetic.  A candidate is decided
// in FP32 only outside a guard band around the threshold; inside it the FP64
// predicate is evaluated with the same operation order and rounding as its
// definition, so the lists are bit-exact.  Lanes farther than kSpanMax cells
// from the reference cell are served in a later pass of the same warp.
//
// Each lane stages its row in shared memory (ordered by position in the cell
// block, then by sorted index); the warp then reserves the rows of the pass
// in the list pool with one atomic add and writes them with coalesced
// stores.  Rows longer than the staging slot are written straight to the
// pool by a second walk over the same candidates.  Row contents are fixed by
// the inputs; only the place of a warp's rows in the pool depends on
// scheduling, and every consumer reads a row through its start and length,
// so all results are bitwise reproducible.  The canonical CSR with prefix
// offsets is built from the pool on demand (sph_get_neighbors).  Nothing
// waits on another warp.
#include "sph_internal.cuh"

namespace sphg {

constexpr int kNbWarps = 2;            // warps per CTA
constexpr int kRowCap = 128;           // staged entries per lane
constexpr int kRowStride = kRowCap + 1;
constexpr int kKeptMax = 64;           // kept-cell batch
constexpr int kSpanMax = 2;            // cells between a lane and the reference cell

struct NbWarpSmem {
    uint32_t rows[32 * kRowStride];    // staged rows, one per lane
    float4 tq[32];                     // candidate tile: position in the reference frame, 4 h^2
    uint32_t tj[32];                   // candidate index
    uint32_t tb[32];                   // candidate cell, packed offset from the reference cell
    uint32_t kst[kKeptMax];            // kept cells: first particle
    uint32_t kpre[kKeptMax];           // kept cells: prefix of the lengths
    uint32_t kb[kKeptMax];             // kept cells: packed offset from the reference cell
};

__device__ __forceinline__ uint32_t pack3(int bx, int by, int bz)
{
    return (uint32_t)(bx + 128) | ((uint32_t)(by + 128) << 8) | ((uint32_t)(bz + 128) << 16);
}

// exact FP64 predicate, no contraction: bit 0 union, bit 1 own radius
__device__ __forceinline__ int exact_pair(double xi, double yi, double zi, double hi, double xj,
                                          double yj, double zj, double hj, double lz)
{
    const double dx = __dsub_rn(xi, xj);
    const double dy = __dsub_rn(yi, yj);
    double dz = __dsub_rn(zi, zj);
    const double hl = __dmul_rn(0.5, lz);
    if (dz > hl) dz = __dsub_rn(dz, lz);
    else if (dz < -hl) dz = __dadd_rn(dz, lz);
    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    const int own = r2 < __dmul_rn(__dmul_rn(4.0, hi), hi);
    const int oth = r2 < __dmul_rn(__dmul_rn(4.0, hj), hj);
    return (own | oth) | (own << 1);
}

__device__ __forceinline__ float warp_min(float v)
{
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float warp_max(float v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// gap between [lo, hi] and the cell [b s, (b+1) s) along one axis
__device__ __forceinline__ float box_gap(float lo, float hi, int b, float s)
{
    const float c0 = (float)b * s, c1 = c0 + s;
    return fmaxf(fmaxf(c0 - hi, lo - c1), 0.0f);
}

struct LaneState {
    float ox, oy, oz;      // particle in the reference frame
    float Ti, flo, fhi;    // 4 h_i^2 and the guard band
    int dx, dy, dz;        // cell offset from the reference cell
    uint32_t kki;          // (dx + 5 dy + 25 dz) << kColBits
    uint32_t cnt, own;
    int64_t i;
    bool act;              // lane takes part in this pass
};

struct WarpBox {
    int refx, refy, refz;
    float x0, y0, z0, x1, y1, z1;  // bounding box of the pass, reference frame
    float hw;                      // largest h of the pass
};

// One walk over the candidates of the lanes in L.act.  DIRECT = false: rows
// are staged in shared memory (up to kRowCap entries); DIRECT = true: lanes
// with direct = true write their whole row to the pool at r0.
template <bool DIRECT>
__device__ void warp_walk(const NbArgs& a, const PatchDev* P, NbWarpSmem& S, LaneState& L, int lane,
                          const WarpBox& B, bool direct, unsigned long long r0)
{
    const float s_f = P->s_f, sz_f = P->sz_f, lz_f = P->lz_f, inv_lz = 1.0f / P->lz_f;
    const int ncx = P->ncx, ncy = P->ncy, ncz = P->ncz, zmode = P->zmode;
    const uint32_t cbase = (uint32_t)P->cell_base;
    const float slack = (1.0f / 4096.0f) * s_f;
    const float Rmax = 2.0f * fmaxf(B.hw, P->hmax_f) * (1.0f + 1.0f / 512.0f) + slack;
    // block of cells around the bounding box, as offsets from the reference cell
    const int xlo = max((int)floorf((B.x0 - Rmax) / s_f), -B.refx);
    const int xhi = min((int)floorf((B.x1 + Rmax) / s_f), ncx - 1 - B.refx);
    const int ylo = max((int)floorf((B.y0 - Rmax) / s_f), -B.refy);
    const int yhi = min((int)floorf((B.y1 + Rmax) / s_f), ncy - 1 - B.refy);
    const int zlo = (int)floorf((B.z0 - Rmax) / sz_f);
    int zhi = (int)floorf((B.z1 + Rmax) / sz_f);
    // a block longer than the period would visit a z cell twice: take one
    // full period instead and the minimum image in FP32
    const bool zwrap = zmode != 0 || (zhi - zlo + 1) >= ncz;
    if (zwrap) zhi = zlo + ncz - 1;
    const int nbx = xhi - xlo + 1, nby = yhi - ylo + 1, nbz = zhi - zlo + 1;
    const int nbox = (nbx > 0 && nby > 0) ? nbx * nby * nbz : 0;
    const unsigned ltmask = (1u << lane) - 1u;
    uint32_t nk = 0, ktot = 0;

    auto flush = [&]() {
        // candidates of the kept batch, 32 per tile
        for (uint32_t fb = 0; fb < ktot; fb += 32) {
            const uint32_t f = fb + lane;
            if (f < ktot) {
                uint32_t c = 0;
                while (c + 1 < nk && S.kpre[c + 1] <= f) c++;
                const uint32_t j = S.kst[c] + (f - S.kpre[c]);
                const uint32_t pb = S.kb[c];
                const float4 q = a.r4[j];
                const int bx = (int)(pb & 255u) - 128, by = (int)((pb >> 8) & 255u) - 128,
                          bz = (int)((pb >> 16) & 255u) - 128;
                S.tq[lane] = make_float4(fmaf((float)bx, s_f, q.x), fmaf((float)by, s_f, q.y),
                                         fmaf((float)bz, sz_f, q.z), q.w);
                // column word for a particle of the reference cell; a lane d cells
                // away subtracts d from the stencil code (exact when |offset| <= 2)
                S.tj[lane] = j | ((uint32_t)((bx + 2) + 5 * (by + 2) + 25 * (bz + 2)) << kColBits);
                S.tb[lane] = pb;
            }
            __syncwarp();
            const uint32_t nt = min(32u, ktot - fb);
            if (L.act) {
                for (uint32_t t = 0; t < nt; t++) {
                    const float4 Q = S.tq[t];
                    const float ex = L.ox - Q.x, ey = L.oy - Q.y;
                    float ez = L.oz - Q.z;
                    // the block may start a whole period away: nearest image
                    if (zwrap) ez = fmaf(-lz_f, rintf(ez * inv_lz), ez);
                    const float r2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
                    const float T = fmaxf(L.Ti, Q.w);
                    if (r2 > T * L.fhi) continue;
                    const uint32_t tw = S.tj[t];
                    const uint32_t j = tw & kColMask;
                    if ((int64_t)j == L.i) continue;
                    bool in = r2 < T * L.flo;
                    bool io = r2 < L.Ti * L.flo;
                    if (!in || (!io && r2 <= L.Ti * L.fhi)) {
                        const int e = exact_pair(a.x[L.i], a.y[L.i], a.z[L.i], a.h[L.i], a.x[j], a.y[j], a.z[j],
                                                 a.h[j], P->lz);
                        in = e & 1;
                        io = (e >> 1) & 1;
                    }
                    L.own += io;
                    if (!in) continue;
                    uint32_t w;
                    if (!zwrap) {
                        w = tw - L.kki;
                    } else {
                        // stencil code of j's cell relative to i's cell, periodic z
                        const uint32_t pb = S.tb[t];
                        const int dcx = (int)(pb & 255u) - 128 - L.dx;
                        const int dcy = (int)((pb >> 8) & 255u) - 128 - L.dy;
                        int dcz = (int)((pb >> 16) & 255u) - 128 - L.dz;
                        int zd;
                        if (zmode == 0) {
                            dcz = ((dcz % ncz) + ncz) % ncz;
                            if (dcz > ncz / 2) dcz -= ncz;
                            zd = dcz + 2;
                        } else {
                            zd = ((dcz % ncz) + ncz) % ncz;
                        }
                        w = j | ((uint32_t)((dcx + 2) + 5 * (dcy + 2) + 25 * zd) << kColBits);
                    }
                    if (DIRECT) {
                        if (direct && r0 + L.cnt < (unsigned long long)a.max_pairs) a.col[r0 + L.cnt] = w;
                    } else if (L.cnt < (uint32_t)kRowCap) {
                        S.rows[lane * kRowStride + L.cnt] = w;
                    }
                    L.cnt++;
                }
            }
            __syncwarp();
        }
        nk = 0;
        ktot = 0;
    };

    for (int cb = 0; cb < nbox; cb += 32) {
        const int c = cb + lane;
        bool keep = false;
        uint32_t st = 0, len = 0, pb = 0;
        if (c < nbox) {
            const int bx = xlo + c % nbx, by = ylo + (c / nbx) % nby, bz = zlo + c / (nbx * nby);
            const int cxj = B.refx + bx, cyj = B.refy + by;
            int czj = (B.refz + bz) % ncz;
            if (czj < 0) czj += ncz;
            const float gz = zwrap ? 0.0f : box_gap(B.z0, B.z1, bz, sz_f);
            const float gx = box_gap(B.x0, B.x1, bx, s_f), gy = box_gap(B.y0, B.y1, by, s_f);
            const float d2 = fmaf(gx, gx, fmaf(gy, gy, gz * gz));
            if (d2 < Rmax * Rmax) {
                const uint32_t lin =
                    cbase + ((uint32_t)czj * (uint32_t)ncy + (uint32_t)cyj) * (uint32_t)ncx + (uint32_t)cxj;
                const uint2 se = a.g.cse[lin];
                if (se.x < se.y) {
                    const float R = 2.0f * fmaxf(B.hw, a.g.chmax[lin]) * (1.0f + 1.0f / 512.0f) + slack;
                    if (d2 < R * R) {
                        keep = true;
                        st = se.x;
                        len = se.y - se.x;
                        pb = pack3(bx, by, bz);
                    }
                }
            }
        }
        uint32_t inc = len;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        const unsigned b = __ballot_sync(0xffffffffu, keep);
        if (keep) {
            const uint32_t k = nk + (uint32_t)__popc(b & ltmask);
            S.kst[k] = st;
            S.kpre[k] = ktot + inc - len;
            S.kb[k] = pb;
        }
        nk += (uint32_t)__popc(b);
        ktot += __shfl_sync(0xffffffffu, inc, 31);
        __syncwarp();
        if (nk > (uint32_t)(kKeptMax - 32) || cb + 32 >= nbox) flush();
    }
}

__global__ void __launch_bounds__(32 * kNbWarps) k_nb_warp(NbArgs a)
{
    extern __shared__ __align__(16) unsigned char nb_smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    NbWarpSmem& S = ((NbWarpSmem*)nb_smem)[warp];
    if (*a.status & kStBad) return;
    for (int64_t q = (int64_t)blockIdx.x * kNbWarps + warp; q < a.nunits; q += (int64_t)gridDim.x * kNbWarps) {
        const WorkItem U = a.units[q];
        const PatchDev* P = a.pd + U.patch;
        const float s_f = P->s_f, sz_f = P->sz_f;
        const int ncz = P->ncz;
        const int64_t i = U.begin + lane;
        const bool valid = i < U.end;
        LaneState L;
        L.i = i;
        float4 r = make_float4(0.f, 0.f, 0.f, 1.f);
        uint32_t cc = 0;
        float hf = 1.0f;
        if (valid) {
            r = a.r4[i];
            cc = a.g.cellxyz[i];
            hf = (float)a.h[i];
        }
        const int cx = cc & 255, cy = (cc >> 8) & 255, cz = cc >> 16;
        const float tol = kTolBase + kTolCell * (s_f / hf);
        L.Ti = r.w;
        L.flo = 1.0f - tol;
        L.fhi = 1.0f + tol;
        unsigned pending = __ballot_sync(0xffffffffu, valid);
        while (pending) {
            // reference cell: the first pending lane; the lanes within kSpanMax
            // cells of it form this pass
            const int ref = __ffs(pending) - 1;
            WarpBox B;
            B.refx = __shfl_sync(0xffffffffu, cx, ref);
            B.refy = __shfl_sync(0xffffffffu, cy, ref);
            B.refz = __shfl_sync(0xffffffffu, cz, ref);
            L.dx = cx - B.refx;
            L.dy = cy - B.refy;
            int dz = cz - B.refz;
            if (dz > ncz / 2) dz -= ncz;
            else if (dz < -(ncz / 2)) dz += ncz;
            L.dz = dz;
            L.kki = (uint32_t)(L.dx + 5 * L.dy + 25 * L.dz) << kColBits;
            L.act = ((pending >> lane) & 1u) && abs(L.dx) <= kSpanMax && abs(L.dy) <= kSpanMax &&
                    abs(L.dz) <= kSpanMax;
            const unsigned actm = __ballot_sync(0xffffffffu, L.act);
            L.ox = fmaf((float)L.dx, s_f, r.x);
            L.oy = fmaf((float)L.dy, s_f, r.y);
            L.oz = fmaf((float)L.dz, sz_f, r.z);
            B.x0 = warp_min(L.act ? L.ox : 3.4e38f);
            B.x1 = warp_max(L.act ? L.ox : -3.4e38f);
            B.y0 = warp_min(L.act ? L.oy : 3.4e38f);
            B.y1 = warp_max(L.act ? L.oy : -3.4e38f);
            B.z0 = warp_min(L.act ? L.oz : 3.4e38f);
            B.z1 = warp_max(L.act ? L.oz : -3.4e38f);
            B.hw = warp_max(L.act ? hf : 0.0f);
            L.cnt = 0;
            L.own = 0;
            warp_walk<false>(a, P, S, L, lane, B, false, 0);
            // reserve the rows of this pass in the pool and write them out
            const uint32_t v = L.act ? L.cnt : 0u;
            uint32_t inc = v;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += t;
            }
            const uint32_t tot = __shfl_sync(0xffffffffu, inc, 31);
            unsigned long long base = 0;
            if (lane == 0) {
                base = atomicAdd(a.pool_used, (unsigned long long)tot);
                if (base + tot > (unsigned long long)a.max_pairs) atomicOr(a.status, kStOverflow);
            }
            base = __shfl_sync(0xffffffffu, base, 0);
            const unsigned long long r0 = base + (inc - v);
            const bool fits = base + tot <= (unsigned long long)a.max_pairs;
            if (L.act) {
                a.rowstart[i] = r0;
                a.cnt[i] = L.cnt;
                a.nown[i] = L.own;
            }
            if (fits) {
                for (int l = 0; l < 32; l++) {
                    if (!((actm >> l) & 1u)) continue;
                    const uint32_t len = min(__shfl_sync(0xffffffffu, L.cnt, l), (uint32_t)kRowCap);
                    const unsigned long long rs = __shfl_sync(0xffffffffu, r0, l);
                    for (uint32_t k = lane; k < len; k += 32) a.col[rs + k] = S.rows[l * kRowStride + k];
                }
                const bool direct = L.act && L.cnt > (uint32_t)kRowCap;
                if (__ballot_sync(0xffffffffu, direct)) {
                    // rows longer than the staging slot: same walk, written to the pool
                    const uint32_t keep_cnt = L.cnt, keep_own = L.own;
                    L.cnt = 0;
                    L.own = 0;
                    warp_walk<true>(a, P, S, L, lane, B, direct, r0);
                    L.cnt = keep_cnt;
                    L.own = keep_own;
                }
            }
            __syncwarp();
            pending &= ~actm;
        }
    }
}

// ---------------------------------------------------------------------------
// Thread-per-particle variant: each lane walks the (2K+1)^3 cells around its
// own cell with its own pruning, in the same loop order as the other lanes of
// its warp (lanes of one cell load the same candidates at the same time), and
// stages its row in shared memory like the warp-tile kernel.
// DIRECT: lanes with direct = true write their whole row to the pool at r0.
// ---------------------------------------------------------------------------
template <bool DIRECT, int K, int ZW>
__device__ uint32_t thread_walk_k(const NbArgs& a, const PatchDev* P, int64_t i, uint32_t* row, bool direct,
                                  unsigned long long r0, uint32_t& own)
{
    constexpr int NX = 2 * K + 1;
    const float s_f = P->s_f, sz_f = P->sz_f, lz_f = P->lz_f, inv_lz = 1.0f / P->lz_f;
    const int ncx = P->ncx, ncy = P->ncy, ncz = P->ncz;
    const uint32_t cbase = (uint32_t)P->cell_base;
    const float4 ri = a.r4[i];
    const uint32_t cc = a.g.cellxyz[i];
    const int cx = cc & 255, cy = (cc >> 8) & 255, cz = cc >> 16;
    const float hf = (float)a.h[i];
    const float Ti = ri.w;
    const float tol = kTolBase + kTolCell * (s_f / hf);
    const float flo = 1.0f - tol, fhi = 1.0f + tol;
    const float slack = (1.0f / 4096.0f) * s_f;
    const float Rg = 2.0f * fmaxf(hf, P->hmax_f) * (1.0f + 1.0f / 512.0f) + slack;
    const float Rg2 = Rg * Rg;
    const float Rc = 2.0f * (1.0f + 1.0f / 512.0f);
    // squared gaps to the cells along x, and their validity, computed once
    float gx2[NX];
    bool vx[NX];
#pragma unroll
    for (int t = 0; t < NX; t++) {
        const int d = t - K;
        const float g = d > 0 ? (float)d * s_f - ri.x : (d < 0 ? ri.x - (float)(d + 1) * s_f : 0.0f);
        const float gg = fmaxf(g, 0.0f);
        gx2[t] = gg * gg;
        vx[t] = (unsigned)(cx + d) < (unsigned)ncx;
    }
    uint32_t cnt = 0;
    const int nz = ZW ? ncz : NX;
    for (int iz = 0; iz < nz; iz++) {
        int czj, zd;
        float zsh, gz2;
        if (!ZW) {
            const int dcz = iz - K;
            czj = cz + dcz;
            if (czj < 0) czj += ncz;
            else if (czj >= ncz) czj -= ncz;
            zsh = (float)dcz * sz_f;
            const float g = dcz > 0 ? (float)dcz * sz_f - ri.z : (dcz < 0 ? ri.z - (float)(dcz + 1) * sz_f : 0.0f);
            const float gg = fmaxf(g, 0.0f);
            gz2 = gg * gg;
            zd = dcz + 2;
        } else {
            czj = cz + iz;
            if (czj >= ncz) czj -= ncz;
            zsh = (float)iz * sz_f;
            gz2 = 0.0f;
            zd = iz;
        }
        if (gz2 >= Rg2) continue;
        const float zo = ri.z - zsh;
        for (int dcy = -K; dcy <= K; dcy++) {
            const int cyj = cy + dcy;
            if ((unsigned)cyj >= (unsigned)ncy) continue;
            const float g = dcy > 0 ? (float)dcy * s_f - ri.y : (dcy < 0 ? ri.y - (float)(dcy + 1) * s_f : 0.0f);
            const float gy = fmaxf(g, 0.0f);
            const float gzy2 = fmaf(gy, gy, gz2);
            if (gzy2 >= Rg2) continue;
            const float yo = ri.y - (float)dcy * s_f;
            const uint32_t lrow = cbase + ((uint32_t)czj * (uint32_t)ncy + (uint32_t)cyj) * (uint32_t)ncx + (uint32_t)cx;
            const uint32_t kkrow = (uint32_t)(2 + 5 * (dcy + 2) + 25 * zd);
#pragma unroll
            for (int t = 0; t < NX; t++) {
                const int dcx = t - K;
                const float d2 = gx2[t] + gzy2;
                if (!vx[t] || d2 >= Rg2) continue;
                const uint32_t lin = lrow + (uint32_t)dcx;
                const uint2 se = a.g.cse[lin];
                const float hc = a.g.chmax[lin];
                if (se.x >= se.y) continue;
                const float R = fmaxf(hf, hc) * Rc + slack;
                if (d2 >= R * R) continue;
                const float xo = ri.x - (float)dcx * s_f;
                const uint32_t kk = (kkrow + (uint32_t)dcx) << kColBits;
                // four candidates per iteration: the gathers are in flight together
                for (uint32_t jb = se.x; jb < se.y; jb += 4) {
                    float4 q[4];
#pragma unroll
                    for (int u = 0; u < 4; u++) q[u] = a.r4[min(jb + (uint32_t)u, se.y - 1u)];
                    float r2[4], T[4];
                    unsigned near = 0;
#pragma unroll
                    for (int u = 0; u < 4; u++) {
                        const float dx = xo - q[u].x, dy = yo - q[u].y;
                        float dz = zo - q[u].z;
                        if (ZW) dz = fmaf(-lz_f, rintf(dz * inv_lz), dz);
                        r2[u] = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                        T[u] = fmaxf(Ti, q[u].w);
                        if (jb + (uint32_t)u < se.y && r2[u] <= T[u] * fhi) near |= 1u << u;
                    }
                    if (!near) continue;
#pragma unroll
                    for (int u = 0; u < 4; u++) {
                        if (!(near & (1u << u))) continue;
                        const uint32_t j = jb + (uint32_t)u;
                        if ((int64_t)j == i) continue;
                        bool in = r2[u] < T[u] * flo;
                        bool io = r2[u] < Ti * flo;
                        if (!in || (!io && r2[u] <= Ti * fhi)) {
                            const int e = exact_pair(a.x[i], a.y[i], a.z[i], a.h[i], a.x[j], a.y[j], a.z[j],
                                                     a.h[j], P->lz);
                            in = e & 1;
                            io = (e >> 1) & 1;
                        }
                        own += io;
                        if (!in) continue;
                        if (DIRECT) {
                            if (direct && r0 + cnt < (unsigned long long)a.max_pairs) a.col[r0 + cnt] = j | kk;
                        } else if (cnt < (uint32_t)kRowCap) {
                            row[cnt] = j | kk;
                        }
                        cnt++;
                    }
                }
            }
        }
    }
    return cnt;
}

template <bool DIRECT>
__device__ __forceinline__ uint32_t thread_walk(const NbArgs& a, const PatchDev* P, int64_t i, uint32_t* row,
                                                bool direct, unsigned long long r0, uint32_t& own)
{
    if (P->zmode) {
        if (P->K == 1) return thread_walk_k<DIRECT, 1, 1>(a, P, i, row, direct, r0, own);
        return thread_walk_k<DIRECT, 2, 1>(a, P, i, row, direct, r0, own);
    }
    if (P->K == 1) return thread_walk_k<DIRECT, 1, 0>(a, P, i, row, direct, r0, own);
    return thread_walk_k<DIRECT, 2, 0>(a, P, i, row, direct, r0, own);
}

__global__ void __launch_bounds__(32 * kNbWarps) k_nb_thread(NbArgs a)
{
    extern __shared__ __align__(16) unsigned char nb_smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    NbWarpSmem& S = ((NbWarpSmem*)nb_smem)[warp];
    if (*a.status & kStBad) return;
    for (int64_t q = (int64_t)blockIdx.x * kNbWarps + warp; q < a.nunits; q += (int64_t)gridDim.x * kNbWarps) {
        const WorkItem U = a.units[q];
        const PatchDev* P = a.pd + U.patch;
        const int64_t i = U.begin + lane;
        const bool act = i < U.end;
        uint32_t cnt = 0, own = 0;
        if (act) cnt = thread_walk<false>(a, P, i, S.rows + lane * kRowStride, false, 0, own);
        const uint32_t v = act ? cnt : 0u;
        uint32_t inc = v;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        const uint32_t tot = __shfl_sync(0xffffffffu, inc, 31);
        unsigned long long base = 0;
        if (lane == 0) {
            base = atomicAdd(a.pool_used, (unsigned long long)tot);
            if (base + tot > (unsigned long long)a.max_pairs) atomicOr(a.status, kStOverflow);
        }
        base = __shfl_sync(0xffffffffu, base, 0);
        const unsigned long long r0 = base + (inc - v);
        const bool fits = base + tot <= (unsigned long long)a.max_pairs;
        if (act) {
            a.rowstart[i] = r0;
            a.cnt[i] = cnt;
            a.nown[i] = own;
        }
        __syncwarp();
        if (fits) {
            const unsigned actm = __ballot_sync(0xffffffffu, act);
            for (int l = 0; l < 32; l++) {
                if (!((actm >> l) & 1u)) continue;
                const uint32_t len = min(__shfl_sync(0xffffffffu, cnt, l), (uint32_t)kRowCap);
                const unsigned long long rs = __shfl_sync(0xffffffffu, r0, l);
                for (uint32_t k = lane; k < len; k += 32) a.col[rs + k] = S.rows[l * kRowStride + k];
            }
            const bool direct = act && cnt > (uint32_t)kRowCap;
            if (direct) {
                uint32_t own2 = 0;
                thread_walk<true>(a, P, i, nullptr, true, r0, own2);
            }
        }
        __syncwarp();
    }
}

int launch_nb_lists(const Launch& L, const NbArgs& a, int tpp)
{
    if (a.n <= 0 || a.nunits <= 0) return 0;
    if (tpp == 1) {
        const size_t smem = sizeof(NbWarpSmem) * kNbWarps;
        static bool attr1 = false;
        if (!attr1) {
            cudaFuncSetAttribute(k_nb_thread, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            attr1 = true;
        }
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_nb_thread, 32 * kNbWarps, smem);
        if (per_sm < 1) per_sm = 1;
        k_nb_thread<<<L.sms * per_sm, 32 * kNbWarps, smem, L.stream>>>(a);
        return 1;
    }
    const size_t smem = sizeof(NbWarpSmem) * kNbWarps;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_nb_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_nb_warp, 32 * kNbWarps, smem);
    if (per_sm < 1) per_sm = 1;
    k_nb_warp<<<L.sms * per_sm, 32 * kNbWarps, smem, L.stream>>>(a);
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
