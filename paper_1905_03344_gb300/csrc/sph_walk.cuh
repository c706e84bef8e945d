// sph_walk.cuh -- the neighbour search of one particle (Table 1 "Neighbour
// Discovery", symmetric union reading R11): j is in N(i) iff j != i and r_ij^2 < 4 h_i^2 or r_ij^2 < 4 h_j^2, with the
// minimum image along periodic z.  n_i = #{j : r_ij^2 < 4 h_i^2} feeds the
// smoothing-length adaptation.
//
// One thread per particle; a warp serves 32 consecutive sorted particles of
// one patch.  The search has up to three parts, each visiting every
// candidate of its kind once:
//   small i, small j: the (2K+1)^3 fine cells around i's cell (template K),
//     pruned by distance against 2 max(h_i, hnb) (hnb: the largest h around
//     i's cell) and then against 2 max(h_i, h_max(cell));
//   big i, small j:   the fine cells within 2 h_i of i (runtime extent);
//   any i, big j:     the 3 x 3 x 3 coarse cells around i's coarse cell
//     (only when the patch has big particles).
// Small particles never reach farther than 2 h_s, and every big one lies in
// the coarse block of any particle it can reach, so the parts together find
// every neighbour exactly once.  A candidate is decided in FP32 only outside
// a guard band around the threshold; inside it the FP64 predicate is
// evaluated with the same operation order and rounding as its definition, so
// the sets are bit-exact.  The walks are templated on the sink that takes
// the decided candidates: the list builder (sph_neighbors.cu) and the
// list-free pair sums (sph_fused.cu) walk the same candidates in the same
// order.
//
// Column word handed to the sink: j | code << 25, code = (dcx+2) + 5 (dcy+2) + 25 zd for a
// neighbour within two fine cells (zd = dcz + 2 with distinct z cells, the z
// cell count offset when all z cells are visited), kFarCode otherwise (the
// pair sums then take the offset from both particles' cell coordinates).
#pragma once
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
static __device__ __noinline__ int exact_pair_at(const NbArgs& a, int64_t i, uint32_t j, double lz)
{
    return exact_pair(a.x[i], a.y[i], a.z[i], a.h[i], a.x[j], a.y[j], a.z[j], a.h[j], lz);
}

#ifndef SPH_NB_MINB
#define SPH_NB_MINB 8                   // resident CTAs per SM the registers are sized for
#endif
#ifndef SPH_NB_GROUP
#define SPH_NB_GROUP 4                  // candidates loaded together per lane (1-5)
#endif
constexpr int kNbtWarps = 4;            // warps per CTA
constexpr int kGroup = SPH_NB_GROUP;
// at most one half of the list ring; the list-free sums' pair queue (eight
// slots) takes a group and three pairs left over, so groups stop at 5
static_assert(kGroup >= 1 && kGroup <= 5, "a group must fit the list ring and the pair queue");
constexpr int kRing = 16;               // ring slots per lane (two halves of 8)
constexpr int kPend = 4;                // guard-band words a ring row defers (per lane)
constexpr uint32_t kHintMargin = 8;     // growth a row may have since the hint, beyond c/3

// Guard band for candidates shifted by up to D cells: the FP32 error of r^2
// grows with the shift (a term of the cell edge per cell), so the cell term
// of the band, sized for shifts of up to 3 cells, scales with D / 3 beyond.
__device__ __forceinline__ float guard_tol(float s_over_h, int D)
{
    return kTolBase + kTolCell * s_over_h * fmaxf(1.0f, (float)D * (1.0f / 3.0f));
}

enum WalkMode { kWalkRing = 0, kWalkFlat = 1 };

// A walk hands every candidate that passed the coarse FP32 test to a sink,
// in groups of at most kGroup candidates:
//   c0 = s.mark();  s.decide(a, P, i, j, r2, Ti, T, flo, fhi, w) ...;  s.group_end(c0);
// with w = j | stencil code << kColBits.  RowSink<MODE> writes the row; the
// list-free pair sums have sinks of their own.

// a candidate that passed the coarse FP32 test r2 <= T (1 + tol): decided in
// FP32 outside the guard band, exactly inside it; bit 0: j in N(i), bit 1:
// within i's own radius
__device__ __forceinline__ int pair_decision(const NbArgs& a, const PatchDev* P, int64_t i, uint32_t j, float r2,
                                             float Ti, float T, float flo, float fhi)
{
    bool in = r2 < T * flo;
    bool io = r2 < Ti * flo;
    if (!in || (!io && r2 <= Ti * fhi)) {
        const int e = exact_pair_at(a, i, j, P->lz);
        in = e & 1;
        io = (e >> 1) & 1;
    }
    return (int)in | ((int)io << 1);
}

__device__ __forceinline__ uint32_t round8(uint32_t v) { return (v + 7u) & ~7u; }

// The list words are written once and read back by the pair sums long after
// (the pool is far larger than L2): they are stored with the streaming hint
// (evict first), so that they do not push the candidate records, which every
// lane re-reads, out of L2.
//
// the row being built by one lane; EXACT = false: every candidate that passed
// the coarse FP32 test (the candidate superset of reused lists), no n_i.
//
// In ring mode the exact FP64 predicate is not evaluated inside the walk: a
// candidate in the guard band is written to the row like a hit and its
// position noted (up to kPend per row, in the lane's slots after its ring),
// and resolve_band() decides those after the walk, removing the ones that
// are no neighbours and counting n_i for the others.  The row is the same as
// with the decision taken in place; the walk's inner loop only holds no call.
// A row with more than kPend such words is walked again with the decisions
// in place (flat mode), as a row that outgrew its reservation is.
template <int MODE, bool EXACT = true>
struct RowSink {
    static constexpr bool kDefer = MODE == kWalkRing && EXACT;
    uint32_t* col;      // the row's first pool entry; flat mode: nullptr = count only
    uint32_t* ring;     // this lane's ring (ring mode): slot k at ring[32 k], then
                        // kPend slots of deferred positions at ring[32 (kRing + k)]
    uint32_t res;       // entries reserved (ring mode)
    uint32_t cnt;       // entries so far
    uint32_t own;       // n_i so far (without the deferred words)
    uint32_t npend;     // guard-band words deferred (ring mode)

    __device__ __forceinline__ void put(uint32_t w)
    {
        if (MODE == kWalkRing) ring[(cnt & (kRing - 1)) * 32] = w;
        else if (col) __stcs(col + cnt, w);
        cnt++;
    }
    __device__ __forceinline__ uint32_t mark() const { return cnt; }
    // after a group of at most 8 puts that started at count c0: at most one
    // half of the ring filled, written out as two 16-byte stores
    __device__ __forceinline__ void group_end(uint32_t c0)
    {
        if (MODE == kWalkRing && ((c0 ^ cnt) & 8u)) {
            const uint32_t blk = c0 & ~7u;
            if (blk + 8u <= res) {
                const uint32_t* rg = ring + ((blk >> 3) & 1u) * (8 * 32);
                uint4* dst = reinterpret_cast<uint4*>(col + blk);
                __stcs(dst, make_uint4(rg[0], rg[32], rg[64], rg[96]));
                __stcs(dst + 1, make_uint4(rg[128], rg[160], rg[192], rg[224]));
            }
        }
    }
    // the partly filled last sector
    __device__ __forceinline__ void finish()
    {
        if (MODE == kWalkRing && cnt <= res)
            for (uint32_t k = cnt & ~7u; k < cnt; k++) __stcs(col + k, ring[(k & (kRing - 1)) * 32]);
    }
    __device__ __forceinline__ void decide(const NbArgs& a, const PatchDev* P, int64_t i, uint32_t j, float r2,
                                           float Ti, float T, float flo, float fhi, uint32_t w)
    {
        if (!EXACT) {
            put(w);
            return;
        }
        if (kDefer) {
            const bool in = r2 < T * flo;
            const bool io = r2 < Ti * flo;
            if (!in || (!io && r2 <= Ti * fhi)) {
                // guard band: kept for now, decided by resolve_band()
                if (npend < (uint32_t)kPend) ring[32 * (kRing + npend)] = cnt;
                npend++;
                put(w);
                return;
            }
            own += (uint32_t)io;
            if (in) put(w);
            return;
        }
        const int d = pair_decision(a, P, i, j, r2, Ti, T, flo, fhi);
        own += (uint32_t)(d >> 1);
        if (d & 1) put(w);
    }
    // after the walk and finish(), with every word in the pool and at most
    // kPend deferred: the exact predicate for each deferred word, last first,
    // so that removing one leaves the positions of the earlier ones valid
    __device__ __forceinline__ void resolve_band(const NbArgs& a, const PatchDev* P, int64_t i)
    {
        for (int k = (int)npend - 1; k >= 0; k--) {
            const uint32_t pos = ring[32 * (kRing + k)];
            const uint32_t j = col[pos] & kColMask;
            const int e = exact_pair_at(a, i, j, P->lz);
            own += (uint32_t)((e >> 1) & 1);
            if (!(e & 1)) {
                for (uint32_t m = pos; m + 1 < cnt; m++) col[m] = col[m + 1];
                cnt--;
            }
        }
        npend = 0;
    }
};

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
template <class S, int K, int ZW>
__device__ __forceinline__ void walk_small(const NbArgs& a, const PatchDev* P, int64_t i, S& row)
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
    // no small neighbour within the stencil has h above hnb of i's cell
    const float hn = a.g.hnb[cbase + ((uint32_t)cz * (uint32_t)ncy + (uint32_t)cy) * (uint32_t)ncx + (uint32_t)cx];
    const float Rg = 2.0f * fmaxf(hf, hn) * (1.0f + 1.0f / 512.0f) + slack;
    const float Rg2 = Rg * Rg;
    const float Rc = 2.0f * (1.0f + 1.0f / 512.0f);
    const float qs = s_f * (1.0f / kBoxQ), qsz = sz_f * (1.0f / kBoxQ);
    // cells more than kr (kz along z) away are farther than Rg: the gap to
    // cell +-d is at least (d - 1) s, and (kr - 1) s > Rg is impossible for
    // kr = floor(Rg / s) + 1 (a relative margin covers the FP32 rounding of
    // the quotient).  The bound is the same on both sides and depends on i
    // only through max(h_i, hnb), so that lanes whose particles share a cell
    // keep walking its stencil in step.
    // (a stencil of at most 2 cells keeps its compile-time bounds)
    const int kr = K <= 2 ? K : min(K, (int)(Rg * P->inv_s_f * (1.0f + 1.0f / 1024.0f)) + 1);
    const int kz = ZW ? 0 : (K <= 2 ? K : min(K, (int)(Rg * P->inv_sz_f * (1.0f + 1.0f / 1024.0f)) + 1));
    const int nz = ZW ? ncz : 2 * kz + 1;
    for (int iz = 0; iz < nz; iz++) {
        int czj, zd;
        float zsh, gz2;
        // raw distance from i to the near z face of the plane (-big: the own plane)
        float gzr = -1e30f;
        uint32_t zshift = 20;
        if (!ZW) {
            const int dcz = iz - kz;
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
        for (int dcy = -kr; dcy <= kr; dcy++) {
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
            // a K = 3 stencil reaches cells 3 away, which have no stencil code
            const bool rowcode = K <= 2 || (dcy >= -2 && dcy <= 2 && zd >= 0 && zd <= 4);
            // one copy of the candidate loop for all x offsets (code size)
#pragma unroll 1
            for (int dcx = -kr; dcx <= kr; dcx++) {
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
                // offsets of up to 2 cells have a stencil code
                const uint32_t kk = (rowcode && dcx >= -2 && dcx <= 2 ? kkrow + (uint32_t)dcx : kFarCode) << kColBits;
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
                    const uint32_t c0 = row.mark();
#pragma unroll
                    for (int u = 0; u < kGroup; u++) {
                        if (!(near & (1u << u))) continue;
                        const uint32_t j = jb + (uint32_t)u;
                        if (j == i32) continue;
                        row.decide(a, P, i, j, r2[u], Ti, T[u], flo, fhi, j | kk);
                    }
                    row.group_end(c0);
                }
            }
        }
    }
}

// ---- big i, small j: the fine cells within 2 h_i of i ---------------------
// (rows pass by value through the out-of-line walks, so that the caller's
// row stays in registers).  Cells are pruned as in walk_small, against their
// tight boxes, and candidates are tested kGroup at a time.
template <class S>
__device__ __noinline__ S walk_big_fine(const NbArgs& a, const PatchDev* P, int64_t i, S row)
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
    const float qs = s_f * (1.0f / kBoxQ), qsz = sz_f * (1.0f / kBoxQ);
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
        // raw distance from i to the near z face of the plane (-big: every z
        // cell visited, or the own plane)
        float gzr = -1e30f;
        uint32_t zshift = 20;
        if (!zw) {
            dcz = iz - Kz;
            czj = ((cz + dcz) % ncz + ncz) % ncz;
            if (dcz != 0) gzr = dcz > 0 ? (float)dcz * sz_f - ri.z : ri.z - (float)(dcz + 1) * sz_f;
            zshift = dcz > 0 ? 20u : 25u;
            const float gg = fmaxf(gzr, 0.0f);
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
            const float gyr = dcy > 0 ? (float)dcy * s_f - ri.y : (dcy < 0 ? ri.y - (float)(dcy + 1) * s_f : -1e30f);
            const uint32_t yshift = dcy > 0 ? 10u : 15u;
            const float gy = fmaxf(gyr, 0.0f);
            const float gzy2 = fmaf(gy, gy, gz2);
            if (gzy2 >= Rg2) continue;
            const float yo = ri.y - (float)dcy * s_f;
            const uint32_t lrow = cbase + ((uint32_t)czj * (uint32_t)ncy + (uint32_t)cyj) * (uint32_t)ncx;
#pragma unroll 1
            for (int dcx = -Kb; dcx <= Kb; dcx++) {
                const int cxj = cx + dcx;
                if ((unsigned)cxj >= (unsigned)ncx) continue;
                const float gxr = dcx > 0 ? (float)dcx * s_f - ri.x : (dcx < 0 ? ri.x - (float)(dcx + 1) * s_f : -1e30f);
                const float gx = fmaxf(gxr, 0.0f);
                const float d2 = fmaf(gx, gx, gzy2);
                if (d2 >= Rg2) continue;
                const uint4 cr = a.g.cell[lrow + (uint32_t)cxj];
                const uint2 se = make_uint2(cr.x, cr.y);
                if (se.x >= se.y) continue;
                const float R = fmaxf(hf, __uint_as_float(cr.z)) * Rc + slack;
                if (tight_gap2(cr.w, gxr, dcx > 0 ? 0u : 5u, gyr, yshift, gzr, zshift, qs, qsz) >= R * R) continue;
                const float xo = ri.x - (float)dcx * s_f;
                const uint32_t kk = stencil_code(P, dcx, dcy, dcz, !zw) << kColBits;
                // kGroup candidates at a time (the record array is padded past
                // its end; slots past the cell are masked)
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
                        if (zw) dz = fmaf(-lz_f, rintf(dz * inv_lz), dz);
                        r2[u] = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                        T[u] = fmaxf(Ti, q[u].w);
                        if ((uint32_t)u < rem && r2[u] <= T[u] * fhi) near |= 1u << u;
                    }
                    if (!near) continue;
                    const uint32_t c0 = row.mark();
#pragma unroll
                    for (int u = 0; u < kGroup; u++) {
                        if (!(near & (1u << u))) continue;
                        const uint32_t j = jb + (uint32_t)u;
                        row.decide(a, P, i, j, r2[u], Ti, T[u], flo, fhi, j | kk);
                    }
                    row.group_end(c0);
                }
            }
        }
    }
    return row;
}

// ---- any i, big j: the coarse cells around i's coarse cell -----------------
template <class S>
__device__ __noinline__ S walk_coarse(const NbArgs& a, const PatchDev* P, int64_t i, S row)
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
                    const uint32_t c0 = row.mark();
                    row.decide(a, P, i, j, r2, Ti, T, flo, fhi, j | kk);
                    row.group_end(c0);
                }
            }
        }
    }
    return row;
}

// the whole search for particle i
template <class S, int K>
__device__ __forceinline__ void walk_all(const NbArgs& a, const PatchDev* P, int64_t i, bool big, S& row)
{
    if (!big) {
        if (P->zmode) walk_small<S, K, 1>(a, P, i, row);
        else walk_small<S, K, 0>(a, P, i, row);
    } else {
        row = walk_big_fine<S>(a, P, i, row);
    }
    if (P->nbig > 0) row = walk_coarse<S>(a, P, i, row);
}

}  // namespace sphg
