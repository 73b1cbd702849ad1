// kp_device.cuh -- per-user device routines of the user pass.
//
//  greedy_walk    Algorithm 1 (Sec. 4.2) in its item-walk form: visit items by
//                 non-increasing cost-adjusted profit p~ (ties: lower index),
//                 accept an item if p~ > 0 and every local set containing it
//                 still has room.  For hierarchical sets this selects exactly
//                 the items Algorithm 1's bottom-up pass keeps.
//  item_thresholds the value theta_j that item j's p~ must exceed for j to be
//                 selected when only p~_j changes (matroid exchange: the best
//                 rejected item j could swap with, or the weakest selected item
//                 in the smallest full set containing j).
//  sweep_k        Map of Algorithm 4 for one (user, k): the k-consumption of
//                 the user's greedy solution as lambda_k falls from +inf to 0,
//                 with the other multipliers fixed.  Instead of re-solving the
//                 greedy at every candidate of Algorithm 3, the sorted order of
//                 the positive lines z_j(lambda_k) is maintained kinetically:
//                 consumption can only change where a line crosses zero or two
//                 adjacent lines swap, and at such an event only the two items
//                 involved can change membership.  Every increase is emitted as
//                 (v1 = lambda_k at the event, v2 = increase).  Used for dense
//                 rows and long CSR rows.
//  exchange_sweep the same map in exchange form (only the events that change
//                 the selection, found from circuit minima), for a few moving
//                 lines; pair_sweep: its straight-line form for two.
//  WindowSink, RefineSink  where the breakpoints go (window masses and
//                 buffer; sub-histogram of a re-run range).
#pragma once
#include <cfloat>
#include <cstdint>

#include "kp_internal.h"

namespace kp {

struct Walk {
    uint64_t sel;   // accepted items
    uint64_t rej;   // positive items rejected by a full set
    uint32_t full;  // sets whose count reached their cap
    uint64_t clo, chi;  // 8-bit counters of sets 0..7 and 8..15
};

__device__ __forceinline__ void walk_add(Walk &w, const Tree &t, int j) {
    w.sel |= 1ull << j;
    uint32_t path = t.ipath[j];
    while (path) {
        int l = __ffs(path) - 1;
        path &= path - 1;
        int sh = 8 * (l & 7);
        uint32_t c;
        if (l < 8) {
            w.clo += 1ull << sh;
            c = (uint32_t)(w.clo >> sh) & 0xffu;
        } else {
            w.chi += 1ull << sh;
            c = (uint32_t)(w.chi >> sh) & 0xffu;
        }
        if (c >= t.cap[l]) w.full |= 1u << l;
    }
}

__device__ __forceinline__ void walk_remove(Walk &w, const Tree &t, int j) {
    w.sel &= ~(1ull << j);
    uint32_t path = t.ipath[j];
    while (path) {
        int l = __ffs(path) - 1;
        path &= path - 1;
        int sh = 8 * (l & 7);
        uint32_t c;
        if (l < 8) {
            w.clo -= 1ull << sh;
            c = (uint32_t)(w.clo >> sh) & 0xffu;
        } else {
            w.chi -= 1ull << sh;
            c = (uint32_t)(w.chi >> sh) & 0xffu;
        }
        if (c < t.cap[l]) w.full &= ~(1u << l);
    }
}

// Greedy over the candidate items `cand` (all must have p~ > 0), reading p~
// from pt[j * ps].
__device__ __forceinline__ void greedy_walk(const float *pt, int ps, uint64_t cand, const Tree &t,
                                            Walk &w) {
    w.sel = 0;
    w.rej = 0;
    w.full = 0;
    w.clo = 0;
    w.chi = 0;
    while (cand) {
        uint64_t r = cand;
        int best = __ffsll((long long)r) - 1;
        float bv = pt[best * ps];
        r &= r - 1;
        while (r) {
            int j = __ffsll((long long)r) - 1;
            r &= r - 1;
            float v = pt[j * ps];
            if (v > bv) {  // strict: the lower index wins ties
                bv = v;
                best = j;
            }
        }
        cand &= ~(1ull << best);
        if (t.ipath[best] & w.full) {
            w.rej |= 1ull << best;
            continue;
        }
        uint32_t before = w.full;
        walk_add(w, t, best);
        uint32_t nf = w.full & ~before;
        if (nf) {  // items blocked by a newly full set can never be accepted
            uint64_t r2 = cand;
            while (r2) {
                int j = __ffsll((long long)r2) - 1;
                r2 &= r2 - 1;
                if (t.ipath[j] & nf) {
                    cand &= ~(1ull << j);
                    w.rej |= 1ull << j;
                }
            }
        }
    }
}

// theta_j for every item given the greedy solution w over all items.
__device__ __forceinline__ void item_thresholds(const float *pt, int M, const Walk &w,
                                                const Tree &t, float *theta) {
    float minSel[KP_MAX_L], maxCut[KP_MAX_L];
    for (int l = 0; l < t.L; ++l) {
        minSel[l] = FLT_MAX;
        maxCut[l] = 0.f;
    }
    uint64_t r = w.sel;
    while (r) {
        int y = __ffsll((long long)r) - 1;
        r &= r - 1;
        float v = pt[y];
        uint32_t path = t.ipath[y];
        while (path) {
            int l = __ffs(path) - 1;
            path &= path - 1;
            minSel[l] = fminf(minSel[l], v);
        }
    }
    r = w.rej;
    while (r) {
        int y = __ffsll((long long)r) - 1;
        r &= r - 1;
        uint32_t f = t.ipath[y] & w.full;
        if (f) {
            int l = __ffs(f) - 1;
            maxCut[l] = fmaxf(maxCut[l], pt[y]);
        }
    }
    for (int j = 0; j < M; ++j) {
        float th = 0.f;
        if ((w.sel >> j) & 1ull) {
            uint32_t path = t.ipath[j];
            while (path) {
                int l = __ffs(path) - 1;
                path &= path - 1;
                th = fmaxf(th, maxCut[l]);
            }
        } else {
            uint32_t f = t.ipath[j] & w.full;
            if (f) th = minSel[__ffs(f) - 1];
        }
        theta[j] = th;
    }
}

// ---------------------------------------------------------------------------
// bucket / key / fixed-point helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t key_of(float v) {
    uint32_t k = __float_as_uint(v);
    return k > 0x7F7FFFFFu ? 0x7F7FFFFFu : k;
}

// Mass of one entry in units of 2^-fixs: round(v * 2^fixs) (to nearest even),
// at most 2^30 for every b of the instance (Params::bscale = 2^fixs): the
// scaling is exact and the conversion is a single 32-bit one.
__device__ __forceinline__ uint32_t bmass(float v, float bscale) {
    return __float2uint_rn(v * bscale);
}

// round(v * 2^s) for finite v >= 0, with integer operations only (on GB300
// the FP64 pipe, which also converts floats to 64-bit integers, is narrow).
// Halves round up.  s is chosen at creation so that no sum can overflow.
__device__ __forceinline__ unsigned long long fixmass(float v, int s) {
    const uint32_t b = __float_as_uint(v);
    const int e = (int)(b >> 23) & 0xff;
    const uint32_t m = e ? ((b & 0x7fffffu) | 0x800000u) : (b & 0x7fffffu);
    const int sh = (e ? e : 1) - 150 + s;  // v = m * 2^((e ? e : 1) - 150)
    if (sh >= 0) return (unsigned long long)m << (sh > 39 ? 39 : sh);
    const int r = -sh;
    if (r > 25) return 0ull;
    return (unsigned long long)((m + (1u << (r - 1))) >> r);
}

// ---------------------------------------------------------------------------
// Map of Algorithm 4 for one (user, k).
//   pt[j*ps]   p~_j at lambda^t;  s[j*ss]  b_jk (0 for items not in J)
//   J          items with b_jk > 0 (the lines that move with lambda_k)
//   lamk       lambda_k^t in FP32
//   w          the greedy selection among the items not in J (the fixed
//              lines): it is the selection at lambda_k = +inf, and no other
//              fixed item can ever enter
// The sorted order of the positive lines is maintained as lambda_k falls;
// only zero crossings and adjacent swaps can change the selection.
// ---------------------------------------------------------------------------
template <int MAXM, class Sink>
__device__ __forceinline__ void sweep_from(const float *pt, int ps, const float *s, int ss, int M,
                                           uint64_t J, float lamk, const Tree &t, int k, Walk w,
                                           Sink &sink) {
    float la[MAXM], ls[MAXM], zc[MAXM], pe[MAXM];
    int ord[MAXM], zl[MAXM];

    int np = 0;
    uint64_t r = w.sel;
    while (r) {  // positive fixed lines, by p~ descending (ties: lower index)
        uint64_t q = r;
        int best = __ffsll((long long)q) - 1;
        float bv = pt[best * ps];
        q &= q - 1;
        while (q) {
            int j = __ffsll((long long)q) - 1;
            q &= q - 1;
            float v = pt[j * ps];
            if (v > bv) {
                bv = v;
                best = j;
            }
        }
        r &= ~(1ull << best);
        la[best] = bv;
        ls[best] = 0.f;
        ord[np++] = best;
    }
    for (int q = 0; q + 1 < np; ++q) pe[q] = -1.f;

    int nz = 0;
    uint64_t mj = J;
    while (mj) {
        int j = __ffsll((long long)mj) - 1;
        mj &= mj - 1;
        float sj = s[j * ss];
        float a = fmaf(lamk, sj, pt[j * ps]);
        la[j] = a;
        ls[j] = sj;
        if (a > 0.f) {
            float z = a / sj;
            zc[j] = z;
            int pos = nz++;  // insertion by zero crossing, descending
            while (pos > 0 && zc[zl[pos - 1]] < z) {
                zl[pos] = zl[pos - 1];
                --pos;
            }
            zl[pos] = j;
        }
    }

    auto pair_ev = [&](int up, int low, float cur) -> float {
        float dsl = ls[low] - ls[up];
        if (!(dsl > 0.f)) return -1.f;
        float x = (la[low] - la[up]) / dsl;
        if (x > cur) x = cur;
        return x > 0.f ? x : -1.f;
    };

    float cur = FLT_MAX;
    int zi = 0;
    const int guard = M * M + 2 * M + 2;
    for (int it = 0; it < guard; ++it) {
        float bs = -1.f;
        int bq = -1;
        for (int q = 0; q + 1 < np; ++q)
            if (pe[q] > bs) {
                bs = pe[q];
                bq = q;
            }
        float bz = zi < nz ? zc[zl[zi]] : -1.f;
        if (bz <= 0.f && bs <= 0.f) break;
        if (bz >= bs) {
            cur = bz;
            int j = zl[zi++];
            ord[np++] = j;
            if (np >= 2) pe[np - 2] = pair_ev(ord[np - 2], j, cur);
            if ((t.ipath[j] & w.full) == 0) {
                walk_add(w, t, j);
                sink.emit(k, cur, ls[j]);
            }
        } else {
            cur = bs;
            int u = ord[bq], v = ord[bq + 1];
            ord[bq] = v;
            ord[bq + 1] = u;
            pe[bq] = -1.f;
            if (bq > 0) pe[bq - 1] = pair_ev(ord[bq - 1], v, cur);
            if (bq + 2 < np) pe[bq + 1] = pair_ev(u, ord[bq + 2], cur);
            if (((w.sel >> u) & 1ull) && !((w.sel >> v) & 1ull)) {
                uint32_t f = t.ipath[v] & w.full;
                if (f) {
                    int tl = __ffs(f) - 1;
                    if ((t.ipath[u] >> tl) & 1u) {
                        walk_remove(w, t, u);
                        walk_add(w, t, v);
                        sink.emit(k, cur, ls[v] - ls[u]);
                    }
                }
            }
        }
    }
}

// Map of Algorithm 4 for one (user, k) in exchange form, for at most JMAX
// moving lines (slots q < nj: item it[q], slope sl[q] = b_jk > 0).
//   pt[j*ps]  p~_j at lambda^t;  S  the selection among the fixed lines at
//   lambda_k = +inf (greedy over the positive items without b_jk)
// Between events the greedy solution S is constant.  As lambda_k falls a
// moving line m outside S gains weight w_m = A_m - lambda_k s_m and enters S
// exactly when w_m exceeds the weakest member of its circuit in S: the
// selected items of the deepest full set on m's path (matroid exchange,
// Proposition 1's structure), or 0 when no set on its path is full.  Fixed
// lines never re-enter once replaced and a moving line leaves S only when a
// moving line with a larger slope overtakes it, so events are few (the loop
// bound is only a guard).  Each event emits (lambda_k at the event, the
// increase of the k-consumption).  The events are the kinetic sweep's consumption
// changes without its swaps of lines that leave S unchanged.  Divisions use
// the fast reciprocal (about 2 ulp; b_jk < 2^100 is checked at creation).
template <int MAXM>
__device__ __forceinline__ float pick(const float (&w)[MAXM], int j) {
    float r = w[0];
#pragma unroll
    for (int q = 1; q < MAXM; ++q) r = j == q ? w[q] : r;
    return r;
}

// w[j] = p~_j at lambda^t (registers, M <= MAXM <= 32)
template <int JMAX, int MAXM, class Sink>
__device__ __forceinline__ void exchange_sweep(const float (&w)[MAXM], uint32_t S, int nj,
                                               const int (&it)[JMAX], const float (&sl)[JMAX],
                                               float lamk, const Tree &t, int k, Sink &sink) {
    float A[JMAX];
    uint32_t Jm = 0u, ipq[JMAX];
#pragma unroll
    for (int q = 0; q < JMAX; ++q) {
        A[q] = q < nj ? fmaf(lamk, sl[q], pick(w, it[q])) : -1.f;
        ipq[q] = q < nj ? t.ipath[it[q]] : 0u;
        if (q < nj) Jm |= 1u << it[q];
    }
    uint32_t inq = 0u, live = 0u;  // slots whose item is in S; slots that can ever enter
#pragma unroll
    for (int q = 0; q < JMAX; ++q)
        if (q < nj && A[q] > 0.f) live |= 1u << q;
    float cur = FLT_MAX;
    const int guard = 8 * nj * nj + 8;
    for (int iter = 0; iter < guard && (live & ~inq); ++iter) {
        uint32_t full = 0u;
        for (int l = 0; l < t.L; ++l)
            if (__popc(S & (uint32_t)t.items[l]) >= (int)t.cap[l]) full |= 1u << l;
        float be = 0.f, bv2 = 0.f;
        int bq = -1;
        uint32_t bout = 0u, brem = 0u;
#pragma unroll
        for (int q = 0; q < JMAX; ++q) {
            if (((live & ~inq) >> q) & 1u) {
                const uint32_t fm = ipq[q] & full;
                float e, v2 = sl[q];
                uint32_t rem = 0u, outq = 0u;
                if (!fm) {
                    e = __fdividef(A[q], sl[q]);  // zero crossing, nothing to replace
                } else {
                    const uint32_t Cm = S & (uint32_t)t.items[__ffs(fm) - 1];
                    const uint32_t CF = Cm & ~Jm;
                    // weakest fixed member (ties: the higher index is weaker)
                    float wmin = FLT_MAX;
                    int y = 0;
#pragma unroll
                    for (int j = 0; j < MAXM; ++j)
                        if (((CF >> j) & 1u) && w[j] <= wmin) {
                            wmin = w[j];
                            y = j;
                        }
                    e = CF ? __fdividef(A[q] - wmin, sl[q]) : -1.f;
                    rem = CF ? 1u << y : 0u;
#pragma unroll
                    for (int r = 0; r < JMAX; ++r) {
                        if (r != q && ((inq >> r) & 1u) && ((Cm >> it[r]) & 1u) && sl[q] > sl[r]) {
                            const float x = __fdividef(A[q] - A[r], sl[q] - sl[r]);
                            if (x > e) {
                                e = x;
                                rem = 1u << it[r];
                                outq = 1u << r;
                                v2 = sl[q] - sl[r];
                            }
                        }
                    }
                }
                if (e > cur) e = cur;
                if (e > be) {
                    be = e;
                    bq = q;
                    brem = rem;
                    bout = outq;
                    bv2 = v2;
                }
            }
        }
        if (bq < 0) break;
        uint32_t add = 0u;
#pragma unroll
        for (int q = 0; q < JMAX; ++q)
            if (q == bq) add = 1u << it[q];
        S = (S & ~brem) | add;
        inq = (inq & ~bout) | (1u << bq);
        cur = be;
        sink.emit(k, be, bv2);
    }
}

// Shortcut of live_sweep below (same arguments, same events): let H = the
// live lines whose zero crossing z is positive and at or above `stop`, R = the
// other live lines positive at lambda_k^t.  If every set l holds
// |SF ∩ l| + |H ∩ l| + [R meets l] <= C_l, no set on the path of a line of H
// is full when it enters and no set on the path of a line of R ever is: the
// lines of H enter at their zero crossings in decreasing order, a line of R
// at its own zero crossing (below `stop`), so the events are exactly
// (z_q, b_q) for q in H.  Returns false, emitting nothing, when the test fails.
template <int MAXM, class Sink>
__device__ __forceinline__ bool live_shortcut(const float *w, uint64_t SF, int nj, const int *it, const float *sl,
                                              float lamk, float stop, const Tree &t, int k, Sink &sink) {
    uint64_t Hm = 0ull, Rm = 0ull;  // items of H and R
    for (int q = 0; q < nj; ++q) {
        const float A = fmaf(lamk, sl[q], w[it[q]]);
        if (A > 0.f) {
            const float z = __fdividef(A, sl[q]);
            if (z > 0.f && z >= stop)
                Hm |= 1ull << it[q];
            else
                Rm |= 1ull << it[q];
        }
    }
    bool fits = true;
    for (int l = 0; l < t.L; ++l) {
        const uint64_t I = t.items[l];
        fits = fits && (__popcll(SF & I) + __popcll(Hm & I) + ((Rm & I) ? 1 : 0) <= (int)t.cap[l]);
    }
    if (!fits) return false;
    for (int q = 0; q < nj; ++q)
        if ((Hm >> it[q]) & 1ull) sink.emit_rel(k, __fdividef(fmaf(lamk, sl[q], w[it[q]]), sl[q]), sl[q]);
    return true;
}

// Map of Algorithm 4 for one (user, k) over the live moving lines only, in
// exchange form, for rows of up to 64 items (dense b).  The live lines (slots
// q < nj, in item order: item it[q], slope sl[q] = b_jk > 0) are the moving
// lines whose zero crossing can reach the pass's floor; any other moving line
// stays negative, hence unselected, at every lambda_k at or above the floor,
// so the events at or above the floor are those of the full sweep, with the
// same arithmetic whatever the floor (every pass computes identical keys).
// SF = the greedy selection among the fixed lines (b_jk = 0), w = the user's
// p~ row.  A line outside S enters when it overtakes the weakest member of its
// circuit in S (the selected items of the deepest full set on its path: the
// weakest fixed line, or a selected moving line with a smaller slope) or, with
// no full set on its path, at its zero crossing; fixed lines never re-enter
// and a moving line leaves only when overtaken, so the events are few (the
// loop bound is a guard).  Each event emits (lambda_k, consumption increase).
// The events come in decreasing lambda_k; the sweep ends at the first one
// below `stop`, a value at or below the pass's floor (the sink drops that
// event and every later one).
template <int MAXM, class Sink>
__device__ void live_sweep(const float *w, uint64_t SF, int nj, const int *it, const float *sl, float lamk,
                           float stop, const Tree &t, int k, Sink &sink) {
    float A[MAXM];
    uint64_t Jm = 0ull, live = 0ull, inq = 0ull;  // items of the live lines; slot masks
    for (int q = 0; q < nj; ++q) {
        A[q] = fmaf(lamk, sl[q], w[it[q]]);
        Jm |= 1ull << it[q];
        if (A[q] > 0.f) live |= 1ull << q;
    }
    uint64_t S = SF;
    float cur = FLT_MAX;
    const int guard = 8 * nj * nj + 8;
    for (int iter = 0; iter < guard && (live & ~inq); ++iter) {
        uint32_t full = 0u;
        for (int l = 0; l < t.L; ++l)
            if (__popcll(S & t.items[l]) >= (int)t.cap[l]) full |= 1u << l;
        float be = 0.f, bv2 = 0.f;
        int bq = -1;
        uint64_t brem = 0ull, bout = 0ull;
        uint64_t cand = live & ~inq;
        int cl = -1;           // circuit level whose weakest fixed member is cached
        float cw = FLT_MAX;
        uint64_t cyb = 0ull;
        while (cand) {
            const int q = __ffsll((long long)cand) - 1;
            cand &= cand - 1;
            const uint32_t fm = t.ipath[it[q]] & full;
            float e, v2 = sl[q];
            uint64_t rem = 0ull, outq = 0ull;
            if (!fm) {
                e = __fdividef(A[q], sl[q]);  // zero crossing, nothing to replace
            } else {
                const int lv = __ffs(fm) - 1;
                const uint64_t Cm = S & t.items[lv];
                if (lv != cl) {
                    // weakest fixed member of the circuit (ties: the higher index is weaker)
                    uint64_t CF = Cm & ~Jm;
                    cw = FLT_MAX;
                    cyb = 0ull;
                    while (CF) {
                        const int j = __ffsll((long long)CF) - 1;
                        CF &= CF - 1;
                        const float v = w[j];
                        if (v <= cw) {
                            cw = v;
                            cyb = 1ull << j;
                        }
                    }
                    cl = lv;
                }
                e = cyb ? __fdividef(A[q] - cw, sl[q]) : -1.f;
                rem = cyb;
                uint64_t mv = inq;  // selected moving members with a smaller slope
                while (mv) {
                    const int r = __ffsll((long long)mv) - 1;
                    mv &= mv - 1;
                    if (((Cm >> it[r]) & 1ull) && sl[q] > sl[r]) {
                        const float x = __fdividef(A[q] - A[r], sl[q] - sl[r]);
                        if (x > e) {
                            e = x;
                            rem = 1ull << it[r];
                            outq = 1ull << r;
                            v2 = sl[q] - sl[r];
                        }
                    }
                }
            }
            if (e > cur) e = cur;
            if (e > be) {
                be = e;
                bq = q;
                brem = rem;
                bout = outq;
                bv2 = v2;
            }
        }
        if (bq < 0 || be < stop) break;
        S = (S & ~brem) | (1ull << it[bq]);
        inq = (inq & ~bout) | (1ull << bq);
        cur = be;
        sink.emit_rel(k, be, bv2);
    }
}

// Sets whose count reached their cap in the selection S.
__device__ __forceinline__ uint32_t full_sets(uint32_t S, const Tree &t) {
    uint32_t full = 0u;
    for (int l = 0; l < t.L; ++l)
        if (__popc(S & (uint32_t)t.items[l]) >= (int)t.cap[l]) full |= 1u << l;
    return full;
}

// Weakest member of the fixed lines CF (ties: the higher index is weaker);
// ybit = its bit (0 if CF is empty).  w = the user's p~ row (shared memory);
// CF holds a few selected items, so the loop visits only them.
__device__ __forceinline__ float weakest(const float *w, uint32_t CF, uint32_t &ybit) {
    float wmin = FLT_MAX;
    uint32_t yb = 0u;
    while (CF) {
        const int j = __ffs(CF) - 1;
        CF &= CF - 1;
        const float v = w[j];
        if (v <= wmin) {
            wmin = v;
            yb = 1u << j;
        }
    }
    ybit = yb;
    return wmin;
}

// lambda_k at which a moving line (weight A - lambda_k s, path ip) enters the
// selection S (full sets `full`), whose circuit holds fixed lines and possibly
// the moving line ob (weight Ao - lambda_k so); rem = the member it replaces.
// Branch-free apart from the short loop over the circuit's fixed members.
__device__ __forceinline__ float entry_time(const float *w, const Tree &t, uint32_t S, uint32_t full,
                                            uint32_t ip, float A, float s, uint32_t ob, float Ao, float so,
                                            uint32_t &rem) {
    const uint32_t fm = ip & full;
    const uint32_t Cm = fm ? S & (uint32_t)t.items[__ffs(fm) - 1] : 0u;
    uint32_t ybit;
    const float wmin = weakest(w, Cm & ~ob, ybit);
    const float ez = __fdividef(A, s);  // zero crossing, nothing to replace
    const float ec = ybit ? __fdividef(A - wmin, s) : -1.f;
    const float ex = ((Cm & ob) && s > so) ? __fdividef(A - Ao, s - so) : -1.f;
    rem = fm ? (ex > ec ? ob : ybit) : 0u;
    return fm ? fmaxf(ec, ex) : ez;
}

// exchange_sweep for exactly two moving lines a, b (slot order a, b), as
// straight-line predicated code: the first line enters, the second enters
// (possibly overtaking the first), and an overtaken first line re-enters; the
// line with the larger slope is never overtaken, so there is no fourth event.
// w = the user's p~ row at lambda^t (shared memory); ki = (lambda_k^t,
// window) of knapsack k.
template <class Sink>
__device__ __forceinline__ void pair_sweep(const float *w, uint32_t SF, int ia, float sa, int ib,
                                           float sb, const float4 &ki, const Tree &t, int k, Sink &sink) {
    const float lamk = ki.x;
    const float Aa = fmaf(lamk, sa, w[ia]), Ab = fmaf(lamk, sb, w[ib]);
    const uint32_t ipa = t.ipath[ia], ipb = t.ipath[ib];
    uint32_t full = full_sets(SF, t), ra, rb;
    float ea = entry_time(w, t, SF, full, ipa, Aa, sa, 0u, 0.f, 0.f, ra);
    float eb = entry_time(w, t, SF, full, ipb, Ab, sb, 0u, 0.f, 0.f, rb);
    ea = Aa > 0.f ? ea : -1.f;
    eb = Ab > 0.f ? eb : -1.f;
    const bool fa = ea >= eb;  // ties: slot a first
    const float e1 = fa ? ea : eb;
    const float Af = fa ? Aa : Ab, sf = fa ? sa : sb, Ao = fa ? Ab : Aa, so = fa ? sb : sa;
    const uint32_t bf = 1u << (fa ? ia : ib), bo = 1u << (fa ? ib : ia);
    const uint32_t ipf = fa ? ipa : ipb, ipo = fa ? ipb : ipa;
    const bool ok1 = e1 > 0.f;
    uint32_t S = (SF & ~(fa ? ra : rb)) | bf;
    full = full_sets(S, t);
    uint32_t ro;
    float e2 = entry_time(w, t, S, full, ipo, Ao, so, bf, Af, sf, ro);
    e2 = fminf(e2, e1);
    const bool ok2 = ok1 && Ao > 0.f && e2 > 0.f;
    const bool over = ok2 && ro == bf;  // the second line overtakes the first
    sink.emit_if(k, ki, e1, sf, ok1);
    sink.emit_if(k, ki, e2, over ? so - sf : so, ok2);
    if (over) {  // rare: a warp skips this unless one of its lanes needs it
        S = (S & ~bf) | bo;
        full = full_sets(S, t);
        uint32_t r3;
        float e3 = entry_time(w, t, S, full, ipf, Af, sf, bo, Ao, so, r3);
        e3 = fminf(e3, e2);
        sink.emit_if(k, ki, e3, sf, e3 > 0.f);
    }
}

// The walk state (counters, full sets) of a given selection.
__device__ __forceinline__ Walk walk_of(uint64_t sel, const Tree &t) {
    Walk w;
    w.sel = 0;
    w.rej = 0;
    w.full = 0;
    w.clo = 0;
    w.chi = 0;
    uint64_t r = sel;
    while (r) {
        const int j = __ffsll((long long)r) - 1;
        r &= r - 1;
        walk_add(w, t, j);
    }
    return w;
}

template <int MAXM, class Sink>
__device__ void sweep_k(const float *pt, int ps, const float *s, int ss, int M, uint64_t J,
                        float lamk, const Tree &t, int k, Sink &sink) {
    uint64_t fcand = 0;
    for (int j = 0; j < M; ++j)
        if (!((J >> j) & 1ull) && pt[j * ps] > 0.f) fcand |= 1ull << j;
    Walk w;
    greedy_walk(pt, ps, fcand, t, w);
    sweep_from<MAXM>(pt, ps, s, ss, M, J, lamk, t, k, w, sink);
}

// ---------------------------------------------------------------------------
// bulk asynchronous copies global -> shared (1-D cp.async.bulk, completion
// counted in bytes on an mbarrier) with bounded waits
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}

// the barriers' initialisation made visible to the asynchronous proxy
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// this thread's earlier generic accesses of shared memory ordered before later
// asynchronous-proxy writes (a buffer refilled after it was read)
__device__ __forceinline__ void fence_proxy_async_shared() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// one arrival that also announces `bytes` of transactions on the barrier
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}

// bytes (a multiple of 16, both addresses 16-byte aligned) from global to
// shared memory, completing `bytes` transactions on bar
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    const unsigned b = (unsigned)__cvta_generic_to_shared(bar);
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(d), "l"(src), "r"(bytes), "r"(b) : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Waits for the phase of the given parity to complete; false after about
// limit_ns nanoseconds (or 2^24 polls) without completion.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
    const uint64_t t0 = global_ns();
    for (int it = 0; it < (1 << 24); ++it) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done) : "r"(a), "r"(parity) : "memory");
        if (done) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
    return false;
}

// ---------------------------------------------------------------------------
// shared-memory atomics through the shared state space (never generic)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t shared_inc_u32(uint32_t *p) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    uint32_t old;
    asm volatile("atom.shared.add.u32 %0, [%1], 1;" : "=r"(old) : "r"(a) : "memory");
    return old;
}

// Exact 64-bit sums in shared memory kept as two 32-bit words per counter: the
// low words lo[0..n) and, n words further, the high words.  A value is added
// to the low word with a native 32-bit atomic; the one addition that wraps the
// low word sees its old value exceed the new one and adds the carry to the high
// word.  The pair therefore holds the exact sum (below 2^64) whatever the
// order of the additions, at the cost of 32-bit atomics only (a 64-bit add to
// shared memory is not a single instruction).
struct SFix {
    uint32_t *lo;  // [2n]: low words, then high words
    int n;
    __device__ __forceinline__ void add(int idx, uint32_t v) const {
        const unsigned a = (unsigned)__cvta_generic_to_shared(lo + idx);
        const unsigned h = a + 4u * (unsigned)n;
        asm volatile("{\n\t.reg .pred c;\n\t.reg .u32 o, t;\n\t"
                     "atom.shared.add.u32 o, [%0], %1;\n\t"
                     "add.u32 t, o, %1;\n\t"
                     "setp.lt.u32 c, t, o;\n\t"
                     "@c red.shared.add.u32 [%2], 1;\n\t}"
                     ::"r"(a), "r"(v), "r"(h) : "memory");
    }
    // add v only where cond != 0 (predicated, no branch)
    __device__ __forceinline__ void add_if(int idx, uint32_t v, uint32_t cond) const {
        const unsigned a = (unsigned)__cvta_generic_to_shared(lo + idx);
        const unsigned h = a + 4u * (unsigned)n;
        asm volatile("{\n\t.reg .pred q, c;\n\t.reg .u32 o, t;\n\t"
                     "setp.ne.u32 q, %3, 0;\n\t"
                     "mov.u32 o, 0;\n\t"
                     "@q atom.shared.add.u32 o, [%0], %1;\n\t"
                     "add.u32 t, o, %1;\n\t"
                     "setp.lt.u32 c, t, o;\n\t"
                     "and.pred c, c, q;\n\t"
                     "@c red.shared.add.u32 [%2], 1;\n\t}"
                     ::"r"(a), "r"(v), "r"(h), "r"(cond) : "memory");
    }
    // a 64-bit value (below 2^63): low half with carry, high half added directly
    __device__ __forceinline__ void add64(int idx, unsigned long long v) const {
        add(idx, (uint32_t)v);
        const uint32_t vh = (uint32_t)(v >> 32);
        if (vh) atomicAdd(lo + n + idx, vh);
    }
    __device__ __forceinline__ unsigned long long get(int idx) const {
        return ((unsigned long long)lo[n + idx] << 32) + lo[idx];
    }
    __device__ __forceinline__ void zero(int idx) const {
        lo[idx] = 0u;
        lo[n + idx] = 0u;
    }
};

// Breakpoint of a knapsack that one item j of the user touches alone:
// lambda_k + (p~_j - theta_j) / b_jk, always rounded the same way (no
// contraction of the addition), so every pass computes identical keys.
__device__ __forceinline__ float breakpoint_value(float lamk, float margin, float b) {
    return __fadd_rn(lamk, __fdividef(margin, b));
}

// ---------------------------------------------------------------------------
// emission sinks
// ---------------------------------------------------------------------------
// First pass: exact masses above / inside / below the window, each split by
// whether the breakpoint lies above lambda_k^t (their sum over the regions is
// the user's k-consumption at lambda^t), and the breakpoints inside the window
// buffered.
struct WindowSink {
    SFix reg6;                 // [3][2][K] (shared): region (above, inside, below the
                               // window) x (v1 > lambda_k^t), knapsack fastest (banks)
    int K;
    const float4 *kinfo;       // [K] (shared): lambda_k (f32), window low, window high (exclusive)
    uint32_t *bcnt;            // [K] buffer fill of this block (shared)
    uint2 *buf;
    int cap_kb, G, blk;
    float bscale;
    // emission of (v1, v2) whose mass m = bmass(v2, bscale) is already known
    __device__ __forceinline__ void emit_km(int k, const float4 &ki, float v1, float v2, uint32_t m) {
        if (!(v1 > 0.f)) return;
        const int r = v1 >= ki.z ? 0 : (v1 >= ki.y ? 1 : 2);
        reg6.add((2 * r + (v1 > ki.x ? 1 : 0)) * K + k, m);
        if (r == 1) {
            const uint32_t slot = shared_inc_u32(&bcnt[k]);
            if (slot < (uint32_t)cap_kb)
                buf[((size_t)k * G + blk) * cap_kb + slot] = make_uint2(key_of(v1), __float_as_uint(v2));
        }
    }
    __device__ __forceinline__ void emit_ki(int k, const float4 &ki, float v1, float v2) {
        emit_km(k, ki, v1, v2, bmass(v2, bscale));
    }
    // bin b = 2 * region + (v1 > lambda_k^t) of a breakpoint with mass m,
    // where emit holds (predicated)
    __device__ __forceinline__ void region_add_if(int k, int b, uint32_t m, bool emit) {
        reg6.add_if(b * K + k, m, emit ? 1u : 0u);
    }
    // predicated emission (pred false: nothing); the buffer append is a rare branch
    __device__ __forceinline__ void emit_if(int k, const float4 &ki, float v1, float v2, bool pred) {
        const bool go = pred && v1 > 0.f && v2 > 0.f;
        const uint32_t m = bmass(v2, bscale);
        const int r = v1 >= ki.z ? 0 : (v1 >= ki.y ? 1 : 2);
        reg6.add_if((2 * r + (v1 > ki.x ? 1 : 0)) * K + k, m, go ? 1u : 0u);
        if (go && r == 1) buffer_add(k, v1, v2);
    }
    // a breakpoint inside the window whose mass region_add_if took
    __device__ __forceinline__ void buffer_add(int k, float v1, float v2) {
        const uint32_t slot = shared_inc_u32(&bcnt[k]);
        if (slot < (uint32_t)cap_kb)
            buf[((size_t)k * G + blk) * cap_kb + slot] = make_uint2(key_of(v1), __float_as_uint(v2));
    }
    __device__ __forceinline__ void emit(int k, float v1, float v2) {
        if (!(v2 > 0.f)) return;
        emit_ki(k, kinfo[k], v1, v2);
    }
    // emission of the dense breakpoint pass: only the window and above are
    // binned (the bins below the window hold each user's total mass instead)
    __device__ __forceinline__ void emit_rel(int k, float v1, float v2) {
        if (!(v1 > 0.f) || !(v2 > 0.f)) return;
        const float4 ki = kinfo[k];
        const int r = v1 >= ki.z ? 0 : (v1 >= ki.y ? 1 : 2);
        if (r == 2) return;
        reg6.add((2 * r) * K + k, bmass(v2, bscale));
        if (r == 1) buffer_add(k, v1, v2);
    }
};

// Bucket of a candidate lambda_k = v around lambda_k^t = lt (Sec. 5.2): with
// d = v - lt, id 0 for |d| < Delta, else sign(d) (1 + floor(log2(|d| / Delta))),
// so the buckets are narrowest at lambda_k^t and double away from it; ids are
// clamped to [-127, 127] and stored at id + 128.  FP32 with IEEE rounding
// (d and |d| / Delta rounded to nearest), floor(log2) from the exponent field.
__device__ __forceinline__ int bucket_index(float v, float lt, float delta) {
    const float d = __fsub_rn(v, lt);
    const float a = __fdiv_rn(fabsf(d), delta);
    int id = 0;
    if (a >= 1.f) {
        const int e = (int)((__float_as_uint(a) >> 23) & 0xffu) - 127;  // a >= 1: normal or inf
        id = 1 + e;
        if (id > 127) id = 127;
        if (d < 0.f) id = -id;
    }
    return id + 128;
}

// Refine pass: sub-histogram of the unresolved range + buffer of its entries.
// A knapsack of a bucketed step (shift -1) bins every breakpoint by its
// bucket around lambda_k^t instead (bucket_index).
struct RefineSink {
    const uint32_t *lo, *hi;      // [K]; empty range for resolved knapsacks
    const int32_t *shift;         // [K]
    const float4 *kinfo;          // [K] (shared): lambda_k^t; bucketed step: Delta_k in .y
    unsigned long long *subhist;  // [K][NSUB] global
    uint32_t *bcnt;               // [K] (shared)
    uint2 *buf;
    int cap_kb, G, blk;
    float bscale;
    __device__ __forceinline__ void emit(int k, float v1, float v2) {
        if (!(v1 > 0.f) || !(v2 > 0.f)) return;
        if (shift[k] < 0) {
            const float4 ki = kinfo[k];
            atomicAdd(&subhist[(size_t)k * NSUB + bucket_index(v1, ki.x, ki.y)],
                      (unsigned long long)bmass(v2, bscale));
            return;
        }
        const uint32_t key = key_of(v1);
        if (key < lo[k] || key >= hi[k]) return;
        const int sb = (int)((key - lo[k]) >> shift[k]);
        atomicAdd(&subhist[(size_t)k * NSUB + sb], (unsigned long long)bmass(v2, bscale));
        const uint32_t slot = shared_inc_u32(&bcnt[k]);
        if (slot < (uint32_t)cap_kb)
            buf[((size_t)k * G + blk) * cap_kb + slot] = make_uint2(key, __float_as_uint(v2));
    }
    __device__ __forceinline__ void emit_ki(int k, const float4 &, float v1, float v2) { emit(k, v1, v2); }
    __device__ __forceinline__ void emit_rel(int k, float v1, float v2) { emit(k, v1, v2); }
    __device__ __forceinline__ void emit_km(int k, const float4 &, float v1, float v2, uint32_t) {
        emit(k, v1, v2);
    }
    __device__ __forceinline__ void region_add_if(int, int, uint32_t, bool) {}
    __device__ __forceinline__ void buffer_add(int, float, float) {}
    __device__ __forceinline__ void emit_if(int k, const float4 &, float v1, float v2, bool pred) {
        if (pred) emit(k, v1, v2);
    }
};

struct NullSink {
    __device__ __forceinline__ void emit(int, float, float) {}
    __device__ __forceinline__ void emit_rel(int, float, float) {}
    __device__ __forceinline__ void emit_ki(int, const float4 &, float, float) {}
    __device__ __forceinline__ void emit_km(int, const float4 &, float, float, uint32_t) {}
    __device__ __forceinline__ void region_add_if(int, int, uint32_t, bool) {}
    __device__ __forceinline__ void buffer_add(int, float, float) {}
    __device__ __forceinline__ void emit_if(int, const float4 &, float, float, bool) {}
};

}  // namespace kp
