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

// the same predicate for sorted slots i, j, out of line: it runs only inside
// the guard band, and one copy keeps the thread walk small
__device__ __noinline__ int exact_pair_at(const NbArgs& a, int64_t i, uint32_t j, double lz)
{
    return exact_pair(a.x[i], a.y[i], a.z[i], a.h[i], a.x[j], a.y[j], a.z[j], a.h[j], lz);
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
                        if (direct && r0 + L.cnt < (unsigned long long)a.pool_cap) a.col[r0 + L.cnt] = w;
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
                base = atomicAdd(&a.pool_used[0], (unsigned long long)tot);
                const unsigned long long before = atomicAdd(&a.pool_used[1], (unsigned long long)tot);
                if (base + tot > (unsigned long long)a.pool_cap || before + tot > (unsigned long long)a.max_pairs)
                    atomicOr(a.status, kStOverflow);
            }
            base = __shfl_sync(0xffffffffu, base, 0);
            const unsigned long long r0 = base + (inc - v);
            const bool fits = base + tot <= (unsigned long long)a.pool_cap;
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
// its warp (lanes of one cell load the same candidates at the same time).
//
// Rows go straight to the pool.  Each lane reserves its row before the walk,
// from the row-length hint c (the particle's row length in the previous
// lists) as c + c/3 + 8 entries -- on a lattice a small change of h adds a
// whole shell of neighbours at once, up to about a third of the row -- or,
// without a hint, from a first walk that only counts.  Reservations are
// rounded up to a multiple of 8 entries, so every row starts on a 32-byte
// boundary.  Hits
// collect in a 16-slot ring in shared memory and leave it as whole 32-byte
// sectors.  A row that outgrows its reservation is walked again into a fresh
// reservation of its exact (rounded) length.  Shared memory per warp is 2 KB,
// which leaves the SM's L1 to the candidate gathers.
// ---------------------------------------------------------------------------
#ifndef SPH_NB_MINB
#define SPH_NB_MINB 8                   // resident CTAs per SM the registers are sized for
#endif
#ifndef SPH_NB_GROUP
#define SPH_NB_GROUP 4                  // candidates loaded together per lane
#endif
constexpr int kNbtWarps = 4;            // warps per CTA
constexpr int kGroup = SPH_NB_GROUP;
static_assert(kGroup >= 1 && kGroup <= 8, "a group may fill at most one half of the ring");
constexpr int kRing = 16;               // ring slots per lane (two halves of 8)
constexpr uint32_t kHintMargin = 8;     // growth a row may have since the hint, beyond c/3

enum WalkMode { kWalkCount = 0, kWalkRing = 1, kWalkDirect = 2 };

struct RowOut {
    uint32_t* col;      // the row's first pool entry
    uint32_t res;       // entries reserved
    uint32_t* ring;     // this lane's ring: slot k at ring[32 k]
};

__device__ __forceinline__ uint32_t round8(uint32_t v) { return (v + 7u) & ~7u; }

// ring half hf (8 entries) to the pool at row entry blk, as two 16-byte stores
__device__ __forceinline__ void ring_flush(const RowOut& o, uint32_t hf, uint32_t blk)
{
    const uint32_t* rg = o.ring + hf * (8 * 32);
    uint4* dst = reinterpret_cast<uint4*>(o.col + blk);
    dst[0] = make_uint4(rg[0], rg[32], rg[64], rg[96]);
    dst[1] = make_uint4(rg[128], rg[160], rg[192], rg[224]);
}

template <int MODE, int K, int ZW>
__device__ uint32_t thread_walk_k(const NbArgs& a, const PatchDev* P, int64_t i, const RowOut& o, uint32_t& own)
{
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
    uint32_t cnt = 0;
    const int nz = ZW ? ncz : 2 * K + 1;
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
            // one copy of the candidate loop for all x offsets (code size)
#pragma unroll 1
            for (int dcx = -K; dcx <= K; dcx++) {
                if ((unsigned)(cx + dcx) >= (unsigned)ncx) continue;
                const float gxr = dcx > 0 ? (float)dcx * s_f - ri.x : (dcx < 0 ? ri.x - (float)(dcx + 1) * s_f : 0.0f);
                const float gx = fmaxf(gxr, 0.0f);
                const float d2 = fmaf(gx, gx, gzy2);
                if (d2 >= Rg2) continue;
                const uint32_t lin = lrow + (uint32_t)dcx;
                const uint2 se = a.g.cse[lin];
                const float hc = a.g.chmax[lin];
                if (se.x >= se.y) continue;
                const float R = fmaxf(hf, hc) * Rc + slack;
                if (d2 >= R * R) continue;
                const float xo = ri.x - (float)dcx * s_f;
                const uint32_t kk = (kkrow + (uint32_t)dcx) << kColBits;
                // kGroup candidates per iteration: their gathers are in flight together
                for (uint32_t jb = se.x; jb < se.y; jb += kGroup) {
                    float4 q[kGroup];
#pragma unroll
                    for (int u = 0; u < kGroup; u++) q[u] = a.r4[min(jb + (uint32_t)u, se.y - 1u)];
                    float r2[kGroup], T[kGroup];
                    unsigned near = 0;
#pragma unroll
                    for (int u = 0; u < kGroup; u++) {
                        const float dx = xo - q[u].x, dy = yo - q[u].y;
                        float dz = zo - q[u].z;
                        if (ZW) dz = fmaf(-lz_f, rintf(dz * inv_lz), dz);
                        r2[u] = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                        T[u] = fmaxf(Ti, q[u].w);
                        if (jb + (uint32_t)u < se.y && r2[u] <= T[u] * fhi) near |= 1u << u;
                    }
                    if (!near) continue;
                    const uint32_t c0 = cnt;
#pragma unroll
                    for (int u = 0; u < kGroup; u++) {
                        if (!(near & (1u << u))) continue;
                        const uint32_t j = jb + (uint32_t)u;
                        if ((int64_t)j == i) continue;
                        bool in = r2[u] < T[u] * flo;
                        bool io = r2[u] < Ti * flo;
                        if (!in || (!io && r2[u] <= Ti * fhi)) {
                            const int e = exact_pair_at(a, i, j, P->lz);
                            in = e & 1;
                            io = (e >> 1) & 1;
                        }
                        own += io;
                        if (!in) continue;
                        if (MODE == kWalkRing) o.ring[(cnt & (kRing - 1)) * 32] = j | kk;
                        else if (MODE == kWalkDirect) o.col[cnt] = j | kk;
                        cnt++;
                    }
                    // at most kGroup <= 8 hits per group: at most one half of the ring filled
                    if (MODE == kWalkRing && ((c0 ^ cnt) & 8u)) {
                        const uint32_t blk = c0 & ~7u;
                        if (blk + 8u <= o.res) ring_flush(o, (blk >> 3) & 1u, blk);
                    }
                }
            }
        }
    }
    if (MODE == kWalkRing && cnt <= o.res) {
        // the partly filled last sector
        const uint32_t blk = cnt & ~7u;
        for (uint32_t k = blk; k < cnt; k++) o.col[k] = o.ring[(k & (kRing - 1)) * 32];
    }
    return cnt;
}

template <int MODE, int K>
__device__ __forceinline__ uint32_t thread_walk(const NbArgs& a, const PatchDev* P, int64_t i, const RowOut& o,
                                                uint32_t& own)
{
    if (P->zmode) return thread_walk_k<MODE, K, 1>(a, P, i, o, own);
    return thread_walk_k<MODE, K, 0>(a, P, i, o, own);
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
        // reservation: the hint plus a margin, or the counted length
        uint32_t res = 0;
        if (act) {
            const uint32_t hint = a.rowcap[i];
            if (hint == kNoHint) {
                uint32_t own0 = 0;
                res = round8(thread_walk<kWalkCount, K>(a, P, i, RowOut{nullptr, 0u, nullptr}, own0));
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
        uint32_t cnt = 0, own = 0;
        if (act) cnt = thread_walk<kWalkRing, K>(a, P, i, RowOut{a.col + r0, ok ? res : 0u, ring}, own);
        if (act && ok && cnt > res) {
            // outgrew the reservation: walk again into an exact one
            const uint32_t need = round8(cnt);
            r0 = atomicAdd(&a.pool_used[0], (unsigned long long)need);
            if (r0 + need <= pool_cap) {
                uint32_t own2 = 0;
                thread_walk<kWalkDirect, K>(a, P, i, RowOut{a.col + r0, need, nullptr}, own2);
            } else {
                atomicOr(a.status, kStOverflow);
            }
        }
        if (act) {
            a.rowstart[i] = r0;
            a.cnt[i] = cnt;
            a.nown[i] = own;
        }
        const uint32_t listed = __shfl_sync(0xffffffffu, warp_incl_scan(act ? cnt : 0u, lane), 31);
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

int launch_nb_lists(const Launch& L, const NbArgs& a, int tpp, int K)
{
    if (a.n <= 0 || a.nunits <= 0) return 0;
    if (tpp == 1) {
        if (K == 1) launch_nb_thread<1>(L, a);
        else launch_nb_thread<2>(L, a);
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
