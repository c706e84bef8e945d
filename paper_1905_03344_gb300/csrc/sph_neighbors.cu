// sph_neighbors.cu -- neighbour discovery, second half: symmetric neighbour
// lists (Table 1 "Neighbour Discovery", symmetric union reading R11): j is
// in N(i) iff j != i and r_ij^2 < 4 h_i^2 or r_ij^2 < 4 h_j^2, with the
// minimum image along periodic z.  n_i = #{j : r_ij^2 < 4 h_i^2} feeds the
// smoothing-length adaptation.
//
// One thread per particle; a warp serves 32 consecutive sorted particles of
// one patch.  The search has up to three parts, each visiting every
// candidate of its kind once:
//   small i, small j: the (2K+1)^3 fine cells around i's cell (template K),
//     pruned by distance against 2 max(h_i, h_max(cell));
//   big i, small j:   the fine cells within 2 h_i of i (runtime extent);
//   any i, big j:     the 3 x 3 x 3 coarse cells around i's coarse cell
//     (only when the patch has big particles).
// Small particles never reach farther than 2 h_s, and every big one lies in
// the coarse block of any particle it can reach, so the parts together find
// every neighbour exactly once.  A candidate is decided in FP32 only outside
// a guard band around the threshold; inside it the FP64 predicate is
// evaluated with the same operation order and rounding as its definition, so
// the lists are bit-exact.
//
// Rows go straight to the pool.  Each lane reserves its row before the walk,
// from the row-length hint c (the particle's row length in the previous
// lists) as c + c/3 + 8 entries -- on a lattice a small change of h adds a
// whole shell of neighbours at once, up to about a third of the row -- or,
// without a hint, from a first walk that only counts.  Reservations are
// rounded up to a multiple of 8 entries, so every row starts on a 32-byte
// boundary.  Hits collect in a 16-slot ring in shared memory and leave it as
// whole 32-byte sectors.  A row that outgrows its reservation is walked again
// into a fresh reservation of its exact (rounded) length.  Shared memory per
// warp is 2 KB, which leaves the SM's L1 to the candidate gathers.  Row
// contents are fixed by the inputs; only the place of a row in the pool
// depends on scheduling, and every consumer reads a row through its start
// and length, so all results are bitwise reproducible.  The canonical CSR
// with prefix offsets is built from the pool on demand (sph_get_neighbors).
//
// Column word: j | code << 25, code = (dcx+2) + 5 (dcy+2) + 25 zd for a
// neighbour within two fine cells (zd = dcz + 2 with distinct z cells, the z
// cell count offset when all z cells are visited), kFarCode otherwise (the
// pair sums then take the offset from both particles' cell coordinates).
#include "sph_internal.cuh"

namespace sphg {

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

// Guard band for candidates shifted by up to D cells: the FP32 error of r^2
// grows with the shift (a term of the cell edge per cell), so the cell term
// of the band, sized for shifts of up to 3 cells, scales with D / 3 beyond.
__device__ __forceinline__ float guard_tol(float s_over_h, int D)
{
    return kTolBase + kTolCell * s_over_h * fmaxf(1.0f, (float)D * (1.0f / 3.0f));
}

enum WalkMode { kWalkRing = 0, kWalkFlat = 1 };

// the row being built by one lane
struct Row {
    uint32_t* col;      // the row's first pool entry; flat mode: nullptr = count only
    uint32_t* ring;     // this lane's ring (ring mode): slot k at ring[32 k]
    uint32_t res;       // entries reserved (ring mode)
    uint32_t cnt;       // entries so far
    uint32_t own;       // n_i so far
};

__device__ __forceinline__ uint32_t round8(uint32_t v) { return (v + 7u) & ~7u; }

template <int MODE>
__device__ __forceinline__ void row_put(Row& r, uint32_t w)
{
    if (MODE == kWalkRing) r.ring[(r.cnt & (kRing - 1)) * 32] = w;
    else if (r.col) r.col[r.cnt] = w;
    r.cnt++;
}

// after a group of at most 8 puts that started at count c0: at most one half
// of the ring filled, written out as two 16-byte stores
template <int MODE>
__device__ __forceinline__ void row_group_end(Row& r, uint32_t c0)
{
    if (MODE == kWalkRing && ((c0 ^ r.cnt) & 8u)) {
        const uint32_t blk = c0 & ~7u;
        if (blk + 8u <= r.res) {
            const uint32_t* rg = r.ring + ((blk >> 3) & 1u) * (8 * 32);
            uint4* dst = reinterpret_cast<uint4*>(r.col + blk);
            dst[0] = make_uint4(rg[0], rg[32], rg[64], rg[96]);
            dst[1] = make_uint4(rg[128], rg[160], rg[192], rg[224]);
        }
    }
}

// the partly filled last sector
template <int MODE>
__device__ __forceinline__ void row_finish(Row& r)
{
    if (MODE == kWalkRing && r.cnt <= r.res)
        for (uint32_t k = r.cnt & ~7u; k < r.cnt; k++) r.col[k] = r.ring[(k & (kRing - 1)) * 32];
}

// a candidate that passed the coarse FP32 test r2 <= T (1 + tol): decide it,
// exactly inside the guard band
template <int MODE>
__device__ __forceinline__ void row_decide(const NbArgs& a, const PatchDev* P, int64_t i, uint32_t j, float r2,
                                           float Ti, float T, float flo, float fhi, uint32_t w, Row& r)
{
    bool in = r2 < T * flo;
    bool io = r2 < Ti * flo;
    if (!in || (!io && r2 <= Ti * fhi)) {
        const int e = exact_pair_at(a, i, j, P->lz);
        in = e & 1;
        io = (e >> 1) & 1;
    }
    r.own += io;
    if (in) row_put<MODE>(r, w);
}

// stencil code of a neighbour at cell offset (dcx, dcy, dcz): dcz is the
// signed offset with distinct z cells (zmode 0, |dcz| <= 2 for a code), the
// z cell count offset modulo ncz when all z cells are visited (zmode 1)
__device__ __forceinline__ uint32_t stencil_code(const PatchDev* P, int dcx, int dcy, int dcz, bool zsigned)
{
    if (dcx < -2 || dcx > 2 || dcy < -2 || dcy > 2) return kFarCode;
    int zd;
    if (P->zmode) {
        zd = dcz % P->ncz;
        if (zd < 0) zd += P->ncz;
        if (zd > 4) return kFarCode;
    } else {
        if (!zsigned || dcz < -2 || dcz > 2) return kFarCode;
        zd = dcz + 2;
    }
    return (uint32_t)((dcx + 2) + 5 * (dcy + 2) + 25 * zd);
}

// squared distance from i to the tight box of a fine cell: g*r are the raw
// distances from i to the cell's near faces (-1e30 along an axis where i is
// inside the cell's slab), the insets come from the cell record at the given
// bit offsets, in units qs = s / kBoxQ (qsz = sz / kBoxQ along z)
__device__ __forceinline__ float tight_gap2(uint32_t box, float gxr, uint32_t xs, float gyr, uint32_t ys, float gzr,
                                            uint32_t zs, float qs, float qsz)
{
    const float tx = fmaxf(fmaf((float)((box >> xs) & 31u), qs, gxr), 0.0f);
    const float ty = fmaxf(fmaf((float)((box >> ys) & 31u), qs, gyr), 0.0f);
    const float tz = fmaxf(fmaf((float)((box >> zs) & 31u), qsz, gzr), 0.0f);
    return fmaf(tx, tx, fmaf(ty, ty, tz * tz));
}

// ---- small i, small j: the (2K+1)^3 fine cells around i's cell ------------
template <int MODE, int K, int ZW>
__device__ __forceinline__ void walk_small(const NbArgs& a, const PatchDev* P, int64_t i, Row& row)
{
    const float s_f = P->s_f, sz_f = P->sz_f, lz_f = P->lz_f, inv_lz = 1.0f / P->lz_f;
    const int ncx = P->ncx, ncy = P->ncy, ncz = P->ncz;
    const uint32_t cbase = (uint32_t)P->cell_base;
    const uint32_t i32 = (uint32_t)i;
    const float4 ri = a.r4[i];
    const uint32_t cc = a.g.cellxyz[i];
    const int cx = cc & 255, cy = (cc >> 8) & 255, cz = cc >> 16;
    const float hf = (float)a.h[i];
    const float Ti = ri.w;
    // every z cell visited (ZW): shifts of up to ncz - 1 cells along z
    const float tol = guard_tol(s_f / hf, ZW ? max(K, ncz) : K);
    const float flo = 1.0f - tol, fhi = 1.0f + tol;
    const float slack = (1.0f / 4096.0f) * s_f;
    const float Rg = 2.0f * fmaxf(hf, P->hs_f) * (1.0f + 1.0f / 512.0f) + slack;
    const float Rg2 = Rg * Rg;
    const float Rc = 2.0f * (1.0f + 1.0f / 512.0f);
    const float qs = s_f * (1.0f / kBoxQ), qsz = sz_f * (1.0f / kBoxQ);
    const int nz = ZW ? ncz : 2 * K + 1;
    for (int iz = 0; iz < nz; iz++) {
        int czj, zd;
        float zsh, gz2;
        // raw distance from i to the near z face of the plane (-big: the own plane)
        float gzr = -1e30f;
        uint32_t zshift = 20;
        if (!ZW) {
            const int dcz = iz - K;
            czj = cz + dcz;
            if (czj < 0) czj += ncz;
            else if (czj >= ncz) czj -= ncz;
            zsh = (float)dcz * sz_f;
            if (dcz != 0) gzr = dcz > 0 ? (float)dcz * sz_f - ri.z : ri.z - (float)(dcz + 1) * sz_f;
            zshift = dcz > 0 ? 20u : 25u;
            const float gg = fmaxf(gzr, 0.0f);
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
            const float gyr = dcy > 0 ? (float)dcy * s_f - ri.y : (dcy < 0 ? ri.y - (float)(dcy + 1) * s_f : -1e30f);
            const uint32_t yshift = dcy > 0 ? 10u : 15u;
            const float gy = fmaxf(gyr, 0.0f);
            const float gzy2 = fmaf(gy, gy, gz2);
            if (gzy2 >= Rg2) continue;
            const float yo = ri.y - (float)dcy * s_f;
            const uint32_t lrow = cbase + ((uint32_t)czj * (uint32_t)ncy + (uint32_t)cyj) * (uint32_t)ncx + (uint32_t)cx;
            const uint32_t kkrow = (uint32_t)(2 + 5 * (dcy + 2) + 25 * zd);
            // one copy of the candidate loop for all x offsets (code size)
#pragma unroll 1
            for (int dcx = -K; dcx <= K; dcx++) {
                if ((unsigned)(cx + dcx) >= (unsigned)ncx) continue;
                const float gxr = dcx > 0 ? (float)dcx * s_f - ri.x : (dcx < 0 ? ri.x - (float)(dcx + 1) * s_f : -1e30f);
                const float gx = fmaxf(gxr, 0.0f);
                const float d2 = fmaf(gx, gx, gzy2);
                if (d2 >= Rg2) continue;
                const uint32_t lin = lrow + (uint32_t)dcx;
                const uint4 cr = a.g.cell[lin];
                const uint2 se = make_uint2(cr.x, cr.y);
                if (se.x >= se.y) continue;
                const float R = fmaxf(hf, __uint_as_float(cr.z)) * Rc + slack;
                if (tight_gap2(cr.w, gxr, dcx > 0 ? 0u : 5u, gyr, yshift, gzr, zshift, qs, qsz) >= R * R) continue;
                const float xo = ri.x - (float)dcx * s_f;
                // offsets of up to 2 cells have a stencil code; K = 3 reaches 3
                const uint32_t kk = (K <= 2 ? kkrow + (uint32_t)dcx
                                            : stencil_code(P, dcx, dcy, ZW ? zd : zd - 2, !ZW)) << kColBits;
                // kGroup candidates per iteration: their gathers are in flight
                // together (the record array has kGroup padding entries, so a
                // group may read past the cell; those slots are masked)
                for (uint32_t jb = se.x; jb < se.y; jb += kGroup) {
                    const float4* qp = a.r4 + jb;
                    float4 q[kGroup];
#pragma unroll
                    for (int u = 0; u < kGroup; u++) q[u] = qp[u];
                    const uint32_t rem = se.y - jb;
                    float r2[kGroup], T[kGroup];
                    unsigned near = 0;
#pragma unroll
                    for (int u = 0; u < kGroup; u++) {
                        const float dx = xo - q[u].x, dy = yo - q[u].y;
                        float dz = zo - q[u].z;
                        if (ZW) dz = fmaf(-lz_f, rintf(dz * inv_lz), dz);
                        r2[u] = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                        T[u] = fmaxf(Ti, q[u].w);
                        if ((uint32_t)u < rem && r2[u] <= T[u] * fhi) near |= 1u << u;
                    }
                    if (!near) continue;
                    const uint32_t c0 = row.cnt;
#pragma unroll
                    for (int u = 0; u < kGroup; u++) {
                        if (!(near & (1u << u))) continue;
                        const uint32_t j = jb + (uint32_t)u;
                        if (j == i32) continue;
                        row_decide<MODE>(a, P, i, j, r2[u], Ti, T[u], flo, fhi, j | kk, row);
                    }
                    row_group_end<MODE>(row, c0);
                }
            }
        }
    }
}

// ---- big i, small j: the fine cells within 2 h_i of i ---------------------
// (rows pass by value through the out-of-line walks, so that the caller's
// row stays in registers)
template <int MODE>
__device__ __noinline__ Row walk_big_fine(const NbArgs& a, const PatchDev* P, int64_t i, Row row)
{
    const float s_f = P->s_f, sz_f = P->sz_f, lz_f = P->lz_f, inv_lz = 1.0f / P->lz_f;
    const int ncx = P->ncx, ncy = P->ncy, ncz = P->ncz;
    const uint32_t cbase = (uint32_t)P->cell_base;
    const float4 ri = a.r4[i];
    const uint32_t cc = a.g.cellxyz[i];
    const int cx = cc & 255, cy = (cc >> 8) & 255, cz = cc >> 16;
    const float hf = (float)a.h[i];
    const float Ti = ri.w;
    const float slack = (1.0f / 4096.0f) * s_f;
    const float Rc = 2.0f * (1.0f + 1.0f / 512.0f);
    const float Rg = fmaxf(hf, P->hs_f) * Rc + slack;
    const float Rg2 = Rg * Rg;
    const int Kb = min((int)ceilf(Rg / s_f), kMaxCellsAxis);
    const int Kz = min((int)ceilf(Rg / sz_f), kMaxCellsAxis);
    // a z block longer than the period: every z cell once, minimum image in FP32
    const bool zw = P->zmode != 0 || 2 * Kz + 1 > ncz;
    const float tol = guard_tol(s_f / hf, max(Kb, zw ? ncz : Kz));
    const float flo = 1.0f - tol, fhi = 1.0f + tol;
    const int nz = zw ? ncz : 2 * Kz + 1;
    for (int iz = 0; iz < nz; iz++) {
        int czj, dcz;
        float gz2 = 0.0f;
        if (!zw) {
            dcz = iz - Kz;
            czj = ((cz + dcz) % ncz + ncz) % ncz;
            const float g = dcz > 0 ? (float)dcz * sz_f - ri.z : (dcz < 0 ? ri.z - (float)(dcz + 1) * sz_f : 0.0f);
            const float gg = fmaxf(g, 0.0f);
            gz2 = gg * gg;
            if (gz2 >= Rg2) continue;
        } else {
            dcz = iz;
            czj = cz + iz;
            if (czj >= ncz) czj -= ncz;
        }
        const float zo = ri.z - (float)dcz * sz_f;
        for (int dcy = -Kb; dcy <= Kb; dcy++) {
            const int cyj = cy + dcy;
            if ((unsigned)cyj >= (unsigned)ncy) continue;
            const float g = dcy > 0 ? (float)dcy * s_f - ri.y : (dcy < 0 ? ri.y - (float)(dcy + 1) * s_f : 0.0f);
            const float gy = fmaxf(g, 0.0f);
            const float gzy2 = fmaf(gy, gy, gz2);
            if (gzy2 >= Rg2) continue;
            const float yo = ri.y - (float)dcy * s_f;
            const uint32_t lrow = cbase + ((uint32_t)czj * (uint32_t)ncy + (uint32_t)cyj) * (uint32_t)ncx;
            for (int dcx = -Kb; dcx <= Kb; dcx++) {
                const int cxj = cx + dcx;
                if ((unsigned)cxj >= (unsigned)ncx) continue;
                const float gxr = dcx > 0 ? (float)dcx * s_f - ri.x : (dcx < 0 ? ri.x - (float)(dcx + 1) * s_f : 0.0f);
                const float gx = fmaxf(gxr, 0.0f);
                const float d2 = fmaf(gx, gx, gzy2);
                if (d2 >= Rg2) continue;
                const uint32_t lin = lrow + (uint32_t)cxj;
                const uint4 cr = a.g.cell[lin];
                const uint2 se = make_uint2(cr.x, cr.y);
                if (se.x >= se.y) continue;
                const float xo = ri.x - (float)dcx * s_f;
                const uint32_t kk = stencil_code(P, dcx, dcy, dcz, !zw) << kColBits;
                for (uint32_t j = se.x; j < se.y; j++) {
                    const float4 q = a.r4[j];
                    const float dx = xo - q.x, dy = yo - q.y;
                    float dz = zo - q.z;
                    if (zw) dz = fmaf(-lz_f, rintf(dz * inv_lz), dz);
                    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    const float T = fmaxf(Ti, q.w);
                    if (r2 > T * fhi) continue;
                    const uint32_t c0 = row.cnt;
                    row_decide<MODE>(a, P, i, j, r2, Ti, T, flo, fhi, j | kk, row);
                    row_group_end<MODE>(row, c0);
                }
            }
        }
    }
    return row;
}

// ---- any i, big j: the coarse cells around i's coarse cell -----------------
template <int MODE>
__device__ __noinline__ Row walk_coarse(const NbArgs& a, const PatchDev* P, int64_t i, Row row)
{
    const float s_f = P->s_f, sz_f = P->sz_f, lz_f = P->lz_f, inv_lz = 1.0f / P->lz_f;
    const int ncx = P->ncx, ncy = P->ncy, ncz = P->ncz;
    const int kc = P->kc, C = 1 << kc;
    const int ncxc = P->ncxc, ncyc = P->ncyc, nczc = P->nczc, zmc = P->zmode_c;
    const float4 ri = a.r4[i];
    const uint32_t cc = a.g.cellxyz[i];
    const int cx = cc & 255, cy = (cc >> 8) & 255, cz = cc >> 16;
    const int X = cx >> kc, Y = cy >> kc, Z = cz >> kc;
    const float hf = (float)a.h[i];
    const float Ti = ri.w;
    const float slack = (1.0f / 4096.0f) * s_f;
    const float Rc = 2.0f * (1.0f + 1.0f / 512.0f);
    const float tol = guard_tol(s_f / hf, 2 * C);
    const float flo = 1.0f - tol, fhi = 1.0f + tol;
    const int nzc = zmc ? nczc : 3;
    for (int iz = 0; iz < nzc; iz++) {
        int Zw, zshift = 0;   // coarse z cell, and the period shift (fine cells) of its image
        float gz = 0.0f;
        if (!zmc) {
            const int Zu = Z + iz - 1;
            Zw = Zu < 0 ? Zu + nczc : (Zu >= nczc ? Zu - nczc : Zu);
            zshift = Zu < 0 ? -ncz : (Zu >= nczc ? ncz : 0);
            const float lo = (float)(Zw * C + zshift - cz) * sz_f;
            const float hi = (float)(min(Zw * C + C, ncz) + zshift - cz) * sz_f;
            gz = fmaxf(fmaxf(lo - ri.z, ri.z - hi), 0.0f);
        } else {
            Zw = iz;
        }
        for (int Yc = max(Y - 1, 0); Yc <= min(Y + 1, ncyc - 1); Yc++) {
            const float ylo = (float)(Yc * C - cy) * s_f, yhi = (float)(min(Yc * C + C, ncy) - cy) * s_f;
            const float gy = fmaxf(fmaxf(ylo - ri.y, ri.y - yhi), 0.0f);
            for (int Xc = max(X - 1, 0); Xc <= min(X + 1, ncxc - 1); Xc++) {
                const float xlo = (float)(Xc * C - cx) * s_f, xhi = (float)(min(Xc * C + C, ncx) - cx) * s_f;
                const float gx = fmaxf(fmaxf(xlo - ri.x, ri.x - xhi), 0.0f);
                const int64_t lin = P->coarse_base + ((int64_t)Zw * ncyc + Yc) * ncxc + Xc;
                const uint4 cr = a.g.cell[lin];
                const uint2 se = make_uint2(cr.x, cr.y);
                if (se.x >= se.y) continue;
                const float R = fmaxf(hf, __uint_as_float(cr.z)) * Rc + slack;
                if (fmaf(gx, gx, fmaf(gy, gy, gz * gz)) >= R * R) continue;
                for (uint32_t j = se.x; j < se.y; j++) {
                    if ((int64_t)j == i) continue;
                    const uint32_t cj = a.g.cellxyz[j];
                    const int dcx = (int)(cj & 255) - cx, dcy = (int)((cj >> 8) & 255) - cy;
                    const int dcz = (int)(cj >> 16) + zshift - cz;
                    const float4 q = a.r4[j];
                    const float dx = (ri.x - (float)dcx * s_f) - q.x;
                    const float dy = (ri.y - (float)dcy * s_f) - q.y;
                    float dz = (ri.z - (float)dcz * sz_f) - q.z;
                    if (zmc) dz = fmaf(-lz_f, rintf(dz * inv_lz), dz);
                    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    const float T = fmaxf(Ti, q.w);
                    if (r2 > T * fhi) continue;
                    const uint32_t kk = stencil_code(P, dcx, dcy, dcz, !zmc) << kColBits;
                    const uint32_t c0 = row.cnt;
                    row_decide<MODE>(a, P, i, j, r2, Ti, T, flo, fhi, j | kk, row);
                    row_group_end<MODE>(row, c0);
                }
            }
        }
    }
    return row;
}

// the whole search for particle i
template <int MODE, int K>
__device__ __forceinline__ void walk_all(const NbArgs& a, const PatchDev* P, int64_t i, bool big, Row& row)
{
    if (!big) {
        if (P->zmode) walk_small<MODE, K, 1>(a, P, i, row);
        else walk_small<MODE, K, 0>(a, P, i, row);
    } else {
        row = walk_big_fine<MODE>(a, P, i, row);
    }
    if (P->nbig > 0) row = walk_coarse<MODE>(a, P, i, row);
}

// counting walk (col = nullptr) and repair walk (straight to the pool): one
// out-of-line copy serves both
template <int K>
__device__ __noinline__ Row walk_all_flat(const NbArgs& a, const PatchDev* P, int64_t i, bool big, Row row)
{
    walk_all<kWalkFlat, K>(a, P, i, big, row);
    return row;
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
        // big particles sit at the end of their patch
        const bool big = act && i >= P->end - (int64_t)P->nbig;
        // reservation: the hint plus a margin, or the counted length
        uint32_t res = 0;
        if (act) {
            const uint32_t hint = a.rowcap[i];
            if (hint == kNoHint) {
                const Row rc = walk_all_flat<K>(a, P, i, big, Row{nullptr, nullptr, 0u, 0u, 0u});
                res = round8(rc.cnt);
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
        Row row = {a.col + r0, ring, ok ? res : 0u, 0u, 0u};
        if (act) {
            walk_all<kWalkRing, K>(a, P, i, big, row);
            row_finish<kWalkRing>(row);
        }
        if (act && ok && row.cnt > res) {
            // outgrew the reservation: walk again into an exact one
            const uint32_t need = round8(row.cnt);
            r0 = atomicAdd(&a.pool_used[0], (unsigned long long)need);
            if (r0 + need <= pool_cap) {
                walk_all_flat<K>(a, P, i, big, Row{a.col + r0, nullptr, need, 0u, 0u});
            } else {
                atomicOr(a.status, kStOverflow);
            }
        }
        if (act) {
            a.rowstart[i] = r0;
            a.cnt[i] = row.cnt;
            a.nown[i] = row.own;
        }
        const uint32_t listed = __shfl_sync(0xffffffffu, warp_incl_scan(act ? row.cnt : 0u, lane), 31);
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

int launch_nb_lists(const Launch& L, const NbArgs& a, int K)
{
    if (a.n <= 0 || a.nunits <= 0) return 0;
    if (K == 1) launch_nb_thread<1>(L, a);
    else if (K == 2) launch_nb_thread<2>(L, a);
    else launch_nb_thread<3>(L, a);
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
