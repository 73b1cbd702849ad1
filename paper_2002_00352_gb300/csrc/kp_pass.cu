// kp_pass.cu -- the per-user pass of dual descent and synchronous coordinate
// descent (Algorithm 2 Map/Reduce, Algorithm 4 Map), one launch per pass over
// all users.
//
// Modes
//   MODE_STATE   reduced costs (Sec. 4.2), Algorithm 1 per user, x bits,
//                consumption R_k = sum_i v_ik (Algorithm 2), dual and primal
//                sums.
//   MODE_HIST    MODE_STATE + Algorithm 4's Map: every user's breakpoints of
//                its k-consumption, aggregated per knapsack into the exact
//                masses above / inside / below a window around the predicted
//                threshold (Sec. 5.2 centres its buckets at lambda_k^t), with
//                the breakpoints inside the window buffered.  A knapsack one
//                item of the user touches has a closed-form breakpoint; two
//                items: pair_sweep from a per-warp queue; three or more:
//                rare_kernel (a launch of its own).
//   MODE_REFINE  Algorithm 4's Map restricted to the key ranges still
//                unresolved by the threshold selection.
//
// Reductions: FP32 per user, exact 64-bit fixed point per knapsack (integer
// atomics, so the result does not depend on the order of the additions),
// 64-bit fixed point for the objective sums too.  The grid is persistent and
// users are assigned to blocks statically, so every sum is reproducible run
// to run.
#include <cstdio>

#include "kp_device.cuh"
#include "kp_internal.h"

namespace kp {

namespace {

constexpr int DENSE_TILE_BYTES = 64 * 1024;   // dense b tile
constexpr int DENSE_USER_BYTES = 96 * 1024;   // all per-user staging of a dense tile

struct SmemLayout {
    size_t lamf, kinfo, bcnt, lo, hi, shift, rfix, reg3, rows, tile_p, tile_b, selm, red, dq;
    size_t tile_p2, tile_b2, bars;  // second stage buffers and their mbarriers (double-buffered pass)
    size_t total;
};

// Per-warp ring of the dense (user, knapsack) tasks whose sweep the shortcut
// does not settle: fewer than 32 wait after each round, 32 more can arrive.
constexpr int DQ_TASKS = 64;
constexpr int DQ_INPLACE = 16;  // lanes of a round from which the sweeps run in place

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

// Per-warp queue of pair sweeps (regular CSR rows): a ring of WQ_OWN owners
// (p~ row, rank masks, user index) and a ring of WQ_TASKS tasks (owner slot,
// first and second entry).  After each round of users fewer than 32 tasks
// wait, so at most 31 + 32 owners and 31 + 96 tasks are ever held.
constexpr int WQ_OWN = 64;
constexpr int WQ_TASKS = 128;
__host__ __device__ inline size_t wq_bytes(int maxm) {
    return align16((size_t)WQ_OWN * (8 * (size_t)maxm + 8) + (size_t)WQ_TASKS * 2);
}

__host__ __device__ inline SmemLayout smem_layout(int layout, int K, int M, int maxm, int threads,
                                                  int T, int mode, int sets = 1, int nbuf = 1) {
    SmemLayout s;
    size_t o = 0;
    s.lamf = o;
    o = align16(o + 4 * (size_t)K);
    s.kinfo = o;
    o = align16(o + 16 * (size_t)K);
    s.bcnt = o;
    o = align16(o + 4 * (size_t)K);
    // refine ranges: re-run passes only
    s.lo = o;
    if (mode == MODE_REFINE) o = align16(o + 4 * (size_t)K);
    s.hi = o;
    if (mode == MODE_REFINE) o = align16(o + 4 * (size_t)K);
    s.shift = o;
    if (mode == MODE_REFINE) o = align16(o + 4 * (size_t)K);
    s.rfix = o;
    o = align16(o + 8 * (size_t)K);
    s.reg3 = o;
    if (mode == MODE_HIST) o = align16(o + (size_t)K * 6 * 8);  // [K][3 regions][2]
    s.red = o;
    o = align16(o + 2 * 8 * 32);
    if (layout == KP_B_CSR) {
        s.rows = o;  // pair-sweep owners' p~ rows and rank masks (register path only: M <= 16):
        // per thread (irregular rows), or per warp a ring of WQ_OWN owners and a
        // ring of WQ_TASKS tasks (regular rows, sets == 0)
        if (mode != MODE_STATE && maxm <= 16)
            o = align16(o + (sets == 0 ? (size_t)(threads / 32) * wq_bytes(maxm) : 2 * 4 * (size_t)threads * maxm));
        s.tile_p = s.tile_b = s.selm = s.dq = o;
        s.tile_p2 = s.tile_b2 = s.bars = o;
    } else {
        s.tile_p = o;
        o = align16(o + 4 * (size_t)T * M);
        s.rows = o;  // p~ of the tile
        o = align16(o + 4 * (size_t)T * M);
        s.selm = o;
        o = align16(o + 8 * (size_t)T);
        s.dq = o;
        if (mode != MODE_STATE) o = align16(o + 4 * (size_t)(threads / 32) * DQ_TASKS);
        s.tile_b = o;
        o = align16(o + 4 * (size_t)T * M * K);
        s.tile_p2 = s.tile_b2 = s.bars = o;
        if (nbuf == 2) {
            s.tile_p2 = o;
            o = align16(o + 4 * (size_t)T * M);
            s.tile_b2 = o;
            o = align16(o + 4 * (size_t)T * M * K);
            s.bars = o;
            o = align16(o + 16);
        }
    }
    s.total = o;
    return s;
}

__device__ __forceinline__ int bitlen(uint32_t x) { return x ? 32 - __clz(x) : 0; }

// Relevance bound of a knapsack (kinfo.w).  A pass needs only the breakpoints
// at or above a floor: in the breakpoint pass of regular CSR rows,
// min(window low, lambda_k^t) (nothing below both is read); in a re-run pass,
// the low end of the unresolved range (+inf when resolved).  A breakpoint
// lambda_k + m / b lies below the floor whenever m < t * b with
//   t = floor - lambda_k - (2^-8 |floor - lambda_k| + 2^-18 (|lambda_k| + |floor|)),
// the margin covering the FP32 rounding of the breakpoint, so such entries are
// skipped without computing them.  Every event of a line is at or below its
// zero crossing lambda_k + p~ / b (the sweeps clamp each event to the
// previous one, the first to a zero crossing or a crossing with a weaker
// selected line), so the same bound with p~ for m skips a whole sweep.
__device__ __forceinline__ float low_bound(float floor_v, float lamk) {
    const float d = floor_v - lamk;
    return d - (0x1p-8f * fabsf(d) + 0x1p-18f * (fabsf(lamk) + fabsf(floor_v)) + 1e-30f);
}

template <int MODE>
__device__ __forceinline__ void init_block_state(const Params &P, const Scratch &S,
                                                 const double *lam, const SmemLayout &L,
                                                 unsigned char *smem, int round, bool leader) {
    const int K = P.K;
    float *lamf = (float *)(smem + L.lamf);
    uint32_t *bcnt = (uint32_t *)(smem + L.bcnt);
    uint32_t *lo = (uint32_t *)(smem + L.lo);
    uint32_t *hi = (uint32_t *)(smem + L.hi);
    int32_t *shift = (int32_t *)(smem + L.shift);
    const SFix rfix{(uint32_t *)(smem + L.rfix), K};
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        float lf = (float)lam[k];
        lamf[k] = lf;
        bcnt[k] = 0;
        rfix.zero(k);
        if (MODE == MODE_HIST) {
            SelK sk = S.sel[k];
            const uint32_t lk = lf > 0.f ? __float_as_uint(lf) : 0u;
            uint32_t c;
            if (sk.pred_key && sk.for_key == lk)  // continuing the trajectory the select predicted
                c = sk.pred_key;
            else
                c = lk ? lk : sk.last_nz_key;
            const long long H = 1ll << sk.w;
            const long long wl = (long long)c - H, wh = (long long)c + H + 1;
            const uint32_t wlo = wl < 1 ? 1u : (uint32_t)wl;
            const uint32_t whi = wh > (long long)KEY_INF ? KEY_INF : (uint32_t)wh;
            if (leader) {
                S.sel[k].ckey = c;
                S.sel[k].wlo = wlo;
                S.sel[k].whi = whi;
            }
            // floor: dense rows read only the window and above (their consumption
            // comes from x, their total from an evaluation at lambda_k = 0);
            // regular CSR rows also need the breakpoints above lambda_k^t
            const float wlf = __uint_as_float(wlo);
            const float fl = P.layout == KP_B_DENSE ? wlf : fminf(wlf, lf);
            // a knapsack outside the block of a block coordinate-descent step
            // gets no breakpoints (its floor is +inf)
            const bool inb = S.block == nullptr || S.block[k] != 0;
            ((float4 *)(smem + L.kinfo))[k] =
                make_float4(lf, wlf, __uint_as_float(whi), inb ? low_bound(fl, lf) : __int_as_float(0x7f800000));
            const SFix r6{(uint32_t *)(smem + L.reg3), 6 * K};
#pragma unroll
            for (int q = 0; q < 6; ++q) r6.zero(q * K + k);
        } else {
            float t = 0.f, dl = 0.f;
            if (MODE == MODE_REFINE) {
                const SelK sk = S.sel[k];
                // a bucketed step reads every positive breakpoint
                t = sk.state == 1   ? low_bound(__uint_as_float(sk.lo), lf)
                    : sk.state == 2 ? low_bound(__uint_as_float(1u), lf)
                                    : __int_as_float(0x7f800000);
                dl = sk.bdelta;
            }
            ((float4 *)(smem + L.kinfo))[k] = make_float4(lf, dl, 0.f, t);
        }
        if (MODE == MODE_REFINE) {
            SelK sk = S.sel[k];
            if (sk.state == 1) {
                lo[k] = sk.lo;
                hi[k] = sk.hi;
                uint32_t width = sk.hi - sk.lo;
                int sh = bitlen(width - 1) - 8;
                shift[k] = sh > 0 ? sh : 0;
            } else if (sk.state == 2) {  // bucketed step: every positive key
                lo[k] = 1u;
                hi[k] = KEY_INF;
                shift[k] = -1;
            } else {
                lo[k] = 0;
                hi[k] = 0;
                shift[k] = 0;
            }
        }
    }
}

// r_from_bins: the consumption R at lambda^t is the mass of the block's
// breakpoints above lambda_k^t (the breakpoint pass of regular CSR rows, which
// takes no explicit consumption); otherwise R was accumulated per entry.
template <int MODE>
__device__ __forceinline__ void flush_block_state(const Params &P, const Scratch &S,
                                                  const SmemLayout &L, unsigned char *smem,
                                                  unsigned long long dsum, unsigned long long psum,
                                                  int blk = -1, bool r_from_bins = false) {
    if (blk < 0) blk = blockIdx.x - S.g_lo;
    const int K = P.K;
    uint32_t *bcnt = (uint32_t *)(smem + L.bcnt);
    const SFix rfix{(uint32_t *)(smem + L.rfix), K};
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        if (MODE != MODE_REFINE) {
            const unsigned long long r = rfix.get(k);
            if (r) atomicAdd(&S.Rfix[k], r);
        }
        if (MODE != MODE_STATE) {
            uint32_t c = bcnt[k];
            S.bufcnt[(size_t)k * S.gspan + blk] = c < (uint32_t)S.cap_kb ? c : (uint32_t)S.cap_kb;
            if (c > (uint32_t)S.cap_kb) S.ovf[k] = 1u;
        }
    }
    if (MODE == MODE_HIST) {
        const SFix r6{(uint32_t *)(smem + L.reg3), 6 * K};
        for (int q = threadIdx.x; q < K * 3; q += blockDim.x) {  // q = 3k + r
            const int k = q / 3, r = q - 3 * k;
            const unsigned long long m = r6.get((2 * r) * K + k) + r6.get((2 * r + 1) * K + k);
            if (m) atomicAdd(&S.reg3[q], m);
        }
        if (r_from_bins)
            for (int k = threadIdx.x; k < K; k += blockDim.x) {
                const unsigned long long m = r6.get(1 * K + k) + r6.get(3 * K + k) + r6.get(5 * K + k);
                if (m) atomicAdd(&S.Rfix[k], m);
            }
    }
    if (MODE != MODE_REFINE) {
        // exact fixed-point objective sums: warp reduction, one atomic per warp
        for (int o = 16; o > 0; o >>= 1) {
            dsum += __shfl_down_sync(0xffffffffu, dsum, o);
            psum += __shfl_down_sync(0xffffffffu, psum, o);
        }
        if ((threadIdx.x & 31) == 0) {
            if (dsum) atomicAdd(&S.objfix[0], dsum);
            if (psum) atomicAdd(&S.objfix[1], psum);
        }
    }
}

__device__ __forceinline__ WindowSink make_window_sink(const Params &P, const Scratch &S,
                                                       const SmemLayout &L, unsigned char *smem) {
    WindowSink ws;
    ws.reg6 = SFix{(uint32_t *)(smem + L.reg3), 6 * P.K};
    ws.K = P.K;
    ws.kinfo = (const float4 *)(smem + L.kinfo);
    ws.bcnt = (uint32_t *)(smem + L.bcnt);
    ws.buf = S.buf;
    ws.cap_kb = S.cap_kb;
    ws.G = S.gspan;
    ws.blk = blockIdx.x - S.g_lo;
    ws.bscale = P.bscale;
    return ws;
}

__device__ __forceinline__ RefineSink make_refine_sink(const Params &P, const Scratch &S,
                                                       const SmemLayout &L, unsigned char *smem) {
    RefineSink rs;
    rs.lo = (const uint32_t *)(smem + L.lo);
    rs.hi = (const uint32_t *)(smem + L.hi);
    rs.shift = (const int32_t *)(smem + L.shift);
    rs.kinfo = (const float4 *)(smem + L.kinfo);
    rs.subhist = S.subhist;
    rs.bcnt = (uint32_t *)(smem + L.bcnt);
    rs.buf = S.buf;
    rs.cap_kb = S.cap_kb;
    rs.G = S.gspan;
    rs.blk = blockIdx.x - S.g_lo;
    rs.bscale = P.bscale;
    return rs;
}

// a[j] for a run-time j without indexing a register array (which would move it
// to local memory): a chain of selects
template <int N>
__device__ __forceinline__ float pick(const float (&a)[N], int j) {
    float r = a[0];
#pragma unroll
    for (int q = 1; q < N; ++q) r = j == q ? a[q] : r;
    return r;
}

// ------------------------------------------------------------------------------------------
// CSR layout: one thread per user, users in tiles of THREADS consecutive users.
// The entry offsets of a tile come from one csr_user_off read plus a block scan
// of the users' entry counts (csr_user_off is consistent with csr_item_nnz,
// checked at creation).  Entries whose knapsack is also consumed by another
// item of the same user are marked once at creation (Scratch::shmask); all
// other entries get the closed-form breakpoint in one uniform loop; knapsacks
// two items share get a pair sweep (per-warp queues; per-thread rows swept after
// every tile when the queues do not fit), those three or
// more share are left to rare_kernel.
// ------------------------------------------------------------------------------------------
template <int THREADS>
__device__ __forceinline__ int block_excl_scan(int v, int *s_scan) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_scan[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int t = lane < THREADS / 32 ? s_scan[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < THREADS / 32) s_scan[lane] = t;
    }
    __syncthreads();
    return (wid > 0 ? s_scan[wid - 1] : 0) + x - v;
}

template <int MAXM, int MODE, class Sink>
__device__ __noinline__ void csr_user(const Params &P, const Scratch &S, int64_t i, int64_t e0,
                                         int nnz, const float *lamf, float *pt, float *mg,
                                         const SFix &rfix, unsigned long long &dsum, unsigned long long &psum,
                                         uint32_t *x_bits, Sink &sink) {
    const int M = P.M;
    const Tree &T = P.tree;
    const float *pr = P.p + (size_t)i * M;
    const uint8_t *nzr = P.innz + (size_t)i * M;
    const float *val = P.val + e0;
    const int16_t *kid = P.kidx + e0;

    // Sec. 4.2: p~_ij = p_ij - sum_k lambda_k b_ijk over the item's entries
    uint64_t pos = 0;
    {
        int e = 0;
        for (int j = 0; j < M; ++j) {
            float acc = __ldg(pr + j);
            const int c = nzr[j];
            for (int q = 0; q < c; ++q, ++e) acc = fmaf(-lamf[kid[e]], __ldg(val + e), acc);
            pt[j] = acc;
            if (acc > 0.f) pos |= 1ull << j;
        }
    }
    // Algorithm 1
    Walk w;
    greedy_walk(pt, 1, pos, T, w);

    if (MODE != MODE_REFINE) {
        if (x_bits)
            for (int q = 0; q < P.W; ++q) x_bits[(size_t)i * P.W + q] = (uint32_t)(w.sel >> (32 * q));
        int e = 0;
        float du = 0.f, pu = 0.f;
        for (int j = 0; j < M; ++j) {
            const int c = nzr[j];
            if ((w.sel >> j) & 1ull) {
                du += pt[j];
                pu += __ldg(pr + j);
                for (int q = 0; q < c; ++q) rfix.add(kid[e + q], bmass(__ldg(val + e + q), P.bscale));
            }
            e += c;
        }
        dsum += fixmass(du, P.fixo);
        psum += fixmass(pu, P.fixo);
    }
    if (MODE == MODE_STATE) return;

    // Algorithm 4 Map.  margin_j = p~_j - theta_j: with a single moving line the
    // breakpoint is lambda_k + margin_j / b_jk.
    item_thresholds(pt, M, w, T, mg);
    for (int j = 0; j < M; ++j) mg[j] = pt[j] - mg[j];
    uint32_t pending = 0;  // first entries of the knapsacks two items use
    if (nnz <= 32) {
        const uint2 shm = S.shmask[i];
        for (int t = 0; t < pair_count(shm.y); ++t) pending |= 1u << pair_first(shm.y, t);
        int e = 0;
        for (int j = 0; j < M; ++j) {
            const int c = nzr[j];
            const float m = mg[j];
            for (int q = 0; q < c; ++q, ++e) {
                if ((shm.x >> e) & 1u) continue;
                const float v = __ldg(val + e);
                if (!(v > 0.f)) continue;
                const int k = kid[e];
                sink.emit(k, breakpoint_value(lamf[k], m, v), v);
            }
        }
    } else {
        // long rows: find shared knapsacks by scanning (no precomputed mask)
        int e = 0;
        for (int j = 0; j < M; ++j) {
            const int c = nzr[j];
            for (int q = 0; q < c; ++q, ++e) {
                const float v = __ldg(val + e);
                if (!(v > 0.f)) continue;
                const int k = kid[e];
                bool shared = false, first = true;
                int f = 0;
                for (int j2 = 0; j2 < M; ++j2) {
                    const int c2 = nzr[j2];
                    if (j2 != j)
                        for (int q2 = 0; q2 < c2; ++q2)
                            if (kid[f + q2] == k && __ldg(val + f + q2) > 0.f) {
                                shared = true;
                                if (f + q2 < e) first = false;
                            }
                    f += c2;
                }
                if (!shared) {
                    sink.emit(k, breakpoint_value(lamf[k], mg[j], v), v);
                } else if (first) {
                    float s[MAXM];
                    uint64_t J = 0;
                    int f2 = 0;
                    for (int j2 = 0; j2 < M; ++j2) {
                        const int c2 = nzr[j2];
                        s[j2] = 0.f;
                        for (int q2 = 0; q2 < c2; ++q2, ++f2)
                            if (kid[f2] == k) {
                                const float vv = __ldg(val + f2);
                                if (vv > 0.f) {
                                    s[j2] = vv;
                                    J |= 1ull << j2;
                                }
                            }
                    }
                    sweep_k<MAXM>(pt, 1, s, 1, M, J, lamf[k], T, k, sink);
                }
            }
        }
    }
    // shared knapsacks: the kinetic sweep, batched after the uniform loop
    while (pending) {
        const int e = __ffs(pending) - 1;
        pending &= pending - 1;
        const int k = kid[e];
        float s[MAXM];
        uint64_t J = 0;
        int f = 0;
        for (int j2 = 0; j2 < M; ++j2) {
            const int c2 = nzr[j2];
            s[j2] = 0.f;
            for (int q2 = 0; q2 < c2; ++q2, ++f)
                if (kid[f] == k) {
                    const float vv = __ldg(val + f);
                    if (vv > 0.f) {
                        s[j2] = vv;
                        J |= 1ull << j2;
                    }
                }
        }
        sweep_k<MAXM>(pt, 1, s, 1, M, J, lamf[k], T, k, sink);
    }
}

// Algorithm 1 in its literal bottom-up form over the candidates cand (items
// with p~ > 0): beats[j] is the set of items ranked before j (larger p~, ties
// to the lower index); at set S_l (deepest first) an item survives if fewer
// than C_l survivors of S_l rank before it.  Registers only (M <= 16).
template <int MAXM>
__device__ __forceinline__ uint32_t greedy_ranked(const float *pt, uint32_t cand, const Tree &T) {
    uint32_t beats[MAXM];
#pragma unroll
    for (int j = 0; j < MAXM; ++j) beats[j] = 0u;
#pragma unroll
    for (int j = 1; j < MAXM; ++j)
#pragma unroll
        for (int j2 = 0; j2 < j; ++j2) {
            const bool first = pt[j2] >= pt[j];  // j2 < j wins ties
            beats[j] |= first ? (1u << j2) : 0u;
            beats[j2] |= first ? 0u : (1u << j);
        }
    uint32_t G = cand;
    for (int l = 0; l < T.L; ++l) {
        const uint32_t inl = G & (uint32_t)T.items[l];
        const int cap = T.cap[l];
        uint32_t drop = 0u;
#pragma unroll
        for (int j = 0; j < MAXM; ++j)
            if (((inl >> j) & 1u) && __popc(beats[j] & inl) >= cap) drop |= 1u << j;
        G &= ~drop;
    }
    return G;
}

// Lean per-user routine for M <= MAXM <= 16 and at most 32 entries: reduced
// costs, decisions and margins live in registers, loops run over the items in
// compile-time order with predication, so the lanes of a warp stay together.
// C > 0: every item has exactly C entries (checked at creation), so entry e
// of the user belongs to item e / C and all entry loops unroll; with
// P.vec the user's rows are read with vector loads.  C = 0: counts are read
// from csr_item_nnz.
//   Algorithm 1 is evaluated in its literal bottom-up form (greedy_ranked).
// Returns the user's list of knapsacks that exactly two of its items use
// (shmask.y: they need a pair sweep); the user's p~ row and positive items
// are then left in prow (and the row after it).
template <int MAXM, int C, int MODE, class Sink>
__device__ __forceinline__ uint32_t csr_user_fast(const Params &P, const Scratch &S, int64_t i,
                                                  int64_t e0, const float *lamf, const float4 *kinfo,
                                                  const SFix &rfix, unsigned long long &dsum,
                                                  unsigned long long &psum, uint32_t *x_bits,
                                                  Sink &sink, float *prow, uint32_t &shared_entries,
                                                  unsigned wmask, float *orow = nullptr, uint32_t *obeat = nullptr,
                                                  unsigned otail = 0u) {
    constexpr int EC = C > 0 ? MAXM * C : 1;
    // breakpoint pass with every entry in registers: the consumption of the
    // selected items is taken in the same predicated loop as the breakpoints
    constexpr bool FOLD = MODE == MODE_HIST && C > 0;
    const int M = P.M;
    const Tree &T = P.tree;
    const float *pr = P.p + (size_t)i * M;
    const uint8_t *nzr = P.innz + (size_t)i * M;
    const float *val = P.val + e0;
    const int16_t *kid = P.kidx + e0;

    float pt[MAXM];
    int cnt[MAXM];
    float vv[EC];
    int kk[EC];
    if constexpr (C > 0) {
        if (P.vec) {  // M == MAXM and the rows are aligned for vector loads
            if constexpr (MAXM % 2 == 0) {
#pragma unroll
                for (int q = 0; q < MAXM / 2; ++q) {
                    const float2 t = __ldg(reinterpret_cast<const float2 *>(pr) + q);
                    pt[2 * q] = t.x;
                    pt[2 * q + 1] = t.y;
                }
            } else {
#pragma unroll
                for (int j = 0; j < MAXM; ++j) pt[j] = __ldg(pr + j);
            }
            if constexpr (EC % 4 == 0) {
#pragma unroll
                for (int q = 0; q < EC / 4; ++q) {
                    const float4 t = __ldg(reinterpret_cast<const float4 *>(val) + q);
                    vv[4 * q] = t.x;
                    vv[4 * q + 1] = t.y;
                    vv[4 * q + 2] = t.z;
                    vv[4 * q + 3] = t.w;
                    const uint2 u = __ldg(reinterpret_cast<const uint2 *>(kid) + q);
                    kk[4 * q] = (int)(int16_t)(u.x & 0xffffu);
                    kk[4 * q + 1] = (int)(int16_t)(u.x >> 16);
                    kk[4 * q + 2] = (int)(int16_t)(u.y & 0xffffu);
                    kk[4 * q + 3] = (int)(int16_t)(u.y >> 16);
                }
            } else {
#pragma unroll
                for (int e = 0; e < EC; ++e) {
                    vv[e] = __ldg(val + e);
                    kk[e] = kid[e];
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < MAXM; ++j) pt[j] = j < M ? __ldg(pr + j) : 0.f;
#pragma unroll
            for (int e = 0; e < EC; ++e) {
                const bool in = e < M * C;
                vv[e] = in ? __ldg(val + e) : 0.f;
                kk[e] = in ? (int)kid[e] : 0;
            }
        }
#pragma unroll
        for (int j = 0; j < MAXM; ++j) cnt[j] = j < M ? C : 0;
    } else {
#pragma unroll
        for (int j = 0; j < MAXM; ++j) {
            pt[j] = j < M ? __ldg(pr + j) : 0.f;
            cnt[j] = j < M ? (int)nzr[j] : 0;
        }
    }
    // Sec. 4.2 reduced costs
    if constexpr (C > 0) {
#pragma unroll
        for (int j = 0; j < MAXM; ++j) {
            float acc = pt[j];
#pragma unroll
            for (int q = 0; q < C; ++q) acc = fmaf(-lamf[kk[j * C + q]], vv[j * C + q], acc);
            pt[j] = acc;
        }
    } else {
        int e = 0;
#pragma unroll
        for (int j = 0; j < MAXM; ++j) {
            float acc = pt[j];
            for (int q = 0; q < cnt[j]; ++q, ++e) acc = fmaf(-lamf[kid[e]], __ldg(val + e), acc);
            pt[j] = acc;
        }
    }
    // Algorithm 1.  A set holding no more positive items than its cap drops
    // none (and neither does any set after it), so the rank masks and the
    // set loop run only for users with some set over its cap.
    uint32_t pos = 0;
#pragma unroll
    for (int j = 0; j < MAXM; ++j)
        if (j < M && pt[j] > 0.f) pos |= 1u << j;
    uint32_t G = pos;
    bool over = false;
    for (int l = 0; l < T.L; ++l) over = over || __popc(pos & (uint32_t)T.items[l]) > (int)T.cap[l];
    if (over) G = greedy_ranked<MAXM>(pt, pos, T);
    uint32_t full = 0u;
    for (int l = 0; l < T.L; ++l)
        if (__popc(G & (uint32_t)T.items[l]) >= (int)T.cap[l]) full |= 1u << l;

    if (MODE != MODE_REFINE) {
        if (x_bits) x_bits[(size_t)i * P.W] = G;
        float du = 0.f, pu = 0.f;
        if constexpr (C > 0) {
#pragma unroll
            for (int j = 0; j < MAXM; ++j) {
                const uint32_t sj = (G >> j) & 1u;
                du += sj ? pt[j] : 0.f;
                pu += sj ? __ldg(pr + j) : 0.f;
                if (!FOLD)
#pragma unroll
                    for (int q = 0; q < C; ++q) rfix.add_if(kk[j * C + q], bmass(vv[j * C + q], P.bscale), sj);
            }
        } else {
            int e = 0;
#pragma unroll
            for (int j = 0; j < MAXM; ++j) {
                if ((G >> j) & 1u) {
                    du += pt[j];
                    pu += __ldg(pr + j);
                    for (int q = 0; q < cnt[j]; ++q) rfix.add(kid[e + q], bmass(__ldg(val + e + q), P.bscale));
                }
                e += cnt[j];
            }
        }
        dsum += fixmass(du, P.fixo);
        psum += fixmass(pu, P.fixo);
    }
    if constexpr (MODE == MODE_STATE) {
        return 0u;
    } else {
        // exchange thresholds theta_j and margins p~_j - theta_j: ts_j = max
        // over the sets on j's path of their best rejected item whose deepest
        // full set it is (j selected), tn_j = the weakest selected item of j's
        // deepest full set.  Only full sets contribute, so the loop visits the
        // full sets, deepest first: the items whose deepest full set is l are
        // those of l that no set visited before holds.
        const uint32_t rej = pos & ~G;
        float ts[MAXM], tn[MAXM];
#pragma unroll
        for (int y = 0; y < MAXM; ++y) {
            ts[y] = 0.f;
            tn[y] = 0.f;
        }
        uint32_t fl = full, cov = 0u;
        while (fl) {
            const int l = __ffs(fl) - 1;
            fl &= fl - 1;
            const uint32_t I = (uint32_t)T.items[l];
            const uint32_t selL = G & I, dyl = I & ~cov, rl = rej & dyl;
            cov |= I;
            float mn = FLT_MAX, mx = 0.f;
#pragma unroll
            for (int j = 0; j < MAXM; ++j) {
                mn = ((selL >> j) & 1u) ? fminf(mn, pt[j]) : mn;
                mx = ((rl >> j) & 1u) ? fmaxf(mx, pt[j]) : mx;
            }
#pragma unroll
            for (int j = 0; j < MAXM; ++j) {
                ts[j] = ((I >> j) & 1u) ? fmaxf(ts[j], mx) : ts[j];
                tn[j] = ((dyl >> j) & 1u) ? mn : tn[j];
            }
        }
        __syncwarp(wmask);
        float mg[MAXM];
#pragma unroll
        for (int j = 0; j < MAXM; ++j) mg[j] = pt[j] - (((G >> j) & 1u) ? ts[j] : tn[j]);
        const uint2 shm = S.shmask[i];
        uint32_t pending = shm.y;
        shared_entries = shm.x;
        if constexpr (FOLD) {
            // Algorithm 4 Map, closed form for knapsacks only one item touches.
            // A cheap first pass marks the entries whose breakpoint can reach a
            // bin the selection reads (m >= t_k b, see low_bound) and the pair
            // entries whose line's zero crossing can (p~ >= t_k b); only the
            // marked entries get the breakpoint, its bin and, inside the
            // window, the buffer.  The consumption at lambda^t is not summed
            // here: it is the mass of the breakpoints above lambda_k^t
            // (flush_block_state), all of them marked (t_k <= 0 < m).
            uint32_t rel = 0u, zrel = 0u;
            float mgl[MAXM];
#pragma unroll
            for (int j = 0; j < MAXM; ++j) mgl[j] = mg[j];
#pragma unroll
            for (int e = 0; e < EC; ++e) {
                const int j = e / C;
                const float v = vv[e];
                const float tv = kinfo[kk[e]].w * v;
                const bool live = v > 0.f;
                rel |= (live && !((shm.x >> e) & 1u) && mg[j] >= tv) ? 1u << e : 0u;
                zrel |= (live && pt[j] >= tv) ? 1u << e : 0u;
            }
            while (rel) {
                const int e = __ffs(rel) - 1;
                rel &= rel - 1;
                const int k = kid[e];
                const float v = __ldg(val + e);
                const float4 ki = kinfo[k];
                const float v1 = breakpoint_value(ki.x, mgl[e / C], v);
                const bool emit = v1 > 0.f;
                const int r = v1 >= ki.z ? 0 : (v1 >= ki.y ? 1 : 2);
                const bool above_t = v1 > ki.x;
                sink.region_add_if(k, 2 * r + (above_t ? 1 : 0), bmass(v, P.bscale), emit && (r != 2 || above_t));
                if (emit && r == 1) sink.buffer_add(k, v1, v);
            }
            // the lanes leave the loop above after different trip counts: meet
            // again before the rest of the user's work (otherwise the warp may
            // run it, and the next users, once per group of lanes)
            __syncwarp(wmask);
            // pairs whose two lines both cross zero below the floor add nothing
            uint32_t kept = 0u;
            int nk = 0;
            for (int t = 0; t < pair_count(pending); ++t) {
                const int e = pair_first(pending, t), e2 = pair_second(pending, t);
                if (((zrel >> e) | (zrel >> e2)) & 1u) {
                    kept |= (uint32_t)((e | (e2 << 5)) << (10 * nk));
                    ++nk;
                }
            }
            pending = nk ? (kept | ((uint32_t)nk << 30)) : 0u;
            __syncwarp(wmask);
        } else {
            // Algorithm 4 Map: closed form for knapsacks only one item touches.
            // One rolled copy of the emission body keeps the code in the
            // instruction cache; entries are re-read from L1.
            int e = 0;
#pragma unroll 1
            for (int j = 0; j < M; ++j) {
                const float m = pick(mg, j);
                const int c = C > 0 ? C : (int)nzr[j];
#pragma unroll 1
                for (int q = 0; q < c; ++q, ++e) {
                    if ((shm.x >> e) & 1u) continue;
                    const int k = kid[e];
                    const float v = __ldg(val + e);
                    if (v > 0.f) {
                        const float4 ki = kinfo[k];
                        // a re-run pass skips breakpoints below its range (low_bound)
                        if (MODE == MODE_REFINE && !(m >= ki.w * v)) continue;
                        sink.emit_ki(k, ki, breakpoint_value(ki.x, m, v), v);
                    }
                }
            }
        }
        uint32_t *brow = nullptr;
        if (orow) {  // the warp's owner ring: slot otail + rank among the lanes with pairs
            const unsigned ob = __ballot_sync(wmask, pending != 0u);
            const unsigned slot = (otail + __popc(ob & ((1u << (threadIdx.x & 31)) - 1u))) & (WQ_OWN - 1);
            prow = orow + slot * MAXM;
            brow = obeat + slot * MAXM;
        } else if (pending) {
            brow = reinterpret_cast<uint32_t *>(prow + (size_t)blockDim.x * MAXM);
        }
        if (pending) {
#pragma unroll
            for (int j = 0; j < MAXM; ++j) prow[j] = pt[j];
            brow[0] = pos;  // the sweep ranks the items again where a cap needs it
        }
        return pending;
    }
}

// One shared-knapsack sweep (a knapsack exactly two items of the owner use,
// entries e and e2, listed at creation; the others have a kernel of their
// own, rare_kernel): the owner's p~ row and rank masks are in shared memory.
template <int MAXM, int C, class Sink>
__device__ __forceinline__ void sweep_task(const Params &P, const float4 *kinfo, const float *prow,
                                           const uint32_t *brow, int64_t i, int64_t e0, int e, int e2,
                                           Sink &sink) {
    const int M = P.M;
    const Tree &T = P.tree;
    const uint8_t *nzr = P.innz + (size_t)i * M;
    const float *val = P.val + e0;
    const int16_t *kid = P.kidx + e0;
    const int k = kid[e];
    const float sa = __ldg(val + e), sb = __ldg(val + e2);
    int ia, ib;
    if constexpr (C > 0) {
        ia = e / C;
        ib = e2 / C;
    } else {
        int acc = 0, j2 = 0;
        while (acc + (int)nzr[j2] <= e) acc += nzr[j2++];
        ia = j2;
        while (acc + (int)nzr[j2] <= e2) acc += nzr[j2++];
        ib = j2;
    }
    const uint32_t J = (1u << ia) | (1u << ib);
    const uint32_t pos = brow[0];
    // selection among the fixed lines: Algorithm 1 over pos minus J (ranked
    // only where a set holds more of them than its cap)
    uint32_t SF = pos & ~J;
    bool over = false;
    for (int l = 0; l < T.L; ++l) over = over || __popc(SF & (uint32_t)T.items[l]) > (int)T.cap[l];
    if (over) {
        float w[MAXM];
#pragma unroll
        for (int j = 0; j < MAXM; ++j) w[j] = prow[j];
        SF = greedy_ranked<MAXM>(w, SF, T);
    }
    pair_sweep(prow, SF, ia, sa, ib, sb, kinfo[k], T, k, sink);
}

// The sweeps of a block's users are pooled and dealt to its threads (about
// 0.8 per thread on the sparse workload), so that the block, which waits for
// its slowest warp, takes one round.  All threads of the block sweep at the
// same time, so the sweep code and the per-user code do not compete for the
// instruction cache.  Called by every thread of the block; contains the block
// barriers that make the owners' rows visible and protect them until done.
// Owner o = u * THREADS + thread is user base + o; with regular rows (C > 0)
// its entries start at uoff0 + (base + o) * M * C, otherwise they are kept.
template <int MAXM, int C, int THREADS, int U, class Sink>
__device__ __forceinline__ void block_sweeps(const Params &P, const float4 *kinfo, float *rows,
                                             int64_t base_user, const int64_t (&ee)[U],
                                             const uint32_t (&pend)[U], Sink &sink) {
    constexpr int QCAP = 2 * U * THREADS;
    constexpr int NW = THREADS / 32;
    constexpr size_t SET = 2 * (size_t)THREADS * MAXM;  // rows of one user set
    static_assert(U * THREADS <= 16384, "task records hold the owner in 14 bits");
    __shared__ uint16_t q[QCAP];
    __shared__ long long we0[C > 0 ? 1 : U * THREADS];
    __shared__ uint32_t wpy[U * THREADS];
    __shared__ int wtot[NW];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int n = 0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
        n += pair_count(pend[u]);
        if (pend[u]) {
            if constexpr (C == 0) we0[u * THREADS + threadIdx.x] = ee[u];
            wpy[u * THREADS + threadIdx.x] = pend[u];
        }
    }
    int x = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wtot[warp] = x;
    __syncthreads();
    int before = 0, total = 0;
#pragma unroll
    for (int w2 = 0; w2 < NW; ++w2) {
        const int t = wtot[w2];
        before += w2 < warp ? t : 0;
        total += t;
    }
    const int base = before + x - n;  // this thread's first slot in the block order
    for (int done = 0; done < total; done += QCAP) {  // the same trip count in every thread
        int slot = base;
#pragma unroll
        for (int u = 0; u < U; ++u)
            for (int t = 0; t < pair_count(pend[u]); ++t, ++slot)
                if (slot >= done && slot < done + QCAP)
                    q[slot - done] = (uint16_t)(((u * THREADS + threadIdx.x) << 2) | t);
        __syncthreads();
        const int nq = total - done < QCAP ? total - done : QCAP;
        for (int t = threadIdx.x; t < nq; t += THREADS) {
            const uint32_t d = q[t];
            const int owner = (int)(d >> 2), pt = (int)(d & 3u);
            const int ou = owner / THREADS, ot = owner - ou * THREADS;
            const float *prow = rows + ou * SET + (size_t)ot * MAXM;
            const uint32_t *brow = reinterpret_cast<const uint32_t *>(prow + (size_t)THREADS * MAXM);
            const uint32_t py = wpy[owner];
            const int64_t oi = base_user + owner;
            const int64_t oe0 = C > 0 ? P.uoff0 + oi * (int64_t)(P.M * C) : we0[C > 0 ? 0 : owner];
            sweep_task<MAXM, C>(P, kinfo, prow, brow, oi, oe0, pair_first(py, pt), pair_second(py, pt), sink);
        }
        __syncthreads();
    }
}

template <int MAXM, int C, int MODE, int THREADS, class Sink>
__device__ __forceinline__ void csr_loop(const Params &P, const Scratch &S, unsigned char *smem,
                                         const SmemLayout &L, uint32_t *x_bits, Sink &sink,
                                         unsigned long long &dsum, unsigned long long &psum, int sets) {
    __shared__ int s_scan[THREADS / 32];
    __shared__ long long s_base;
    const int M = P.M;
    const float *lamf = (const float *)(smem + L.lamf);
    const float4 *kinfo = (const float4 *)(smem + L.kinfo);
    const SFix rfix{(uint32_t *)(smem + L.rfix), P.K};
    float *rows = (float *)(smem + L.rows);
    if constexpr (C > 0 && MODE != MODE_STATE && MAXM <= 16) if (sets == 0) {
        // regular rows: each warp queues its users' pair sweeps and sweeps 32 of
        // them at a time, so the loop has no block barrier and every sweep round
        // is full
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        unsigned char *wq = smem + L.rows + (size_t)warp * wq_bytes(MAXM);
        float *orow = (float *)wq;                                      // [WQ_OWN][MAXM]
        uint32_t *obeat = (uint32_t *)(orow + WQ_OWN * MAXM);            // [WQ_OWN][MAXM]
        long long *ouser = (long long *)(obeat + WQ_OWN * MAXM);         // [WQ_OWN]
        uint16_t *tq = (uint16_t *)(ouser + WQ_OWN);                     // [WQ_TASKS]
        unsigned head = 0u, tail = 0u, otail = 0u;                       // the same in every lane
        const unsigned lt = (1u << lane) - 1u;
        auto round = [&](int ntask) {
            if (lane < ntask) {
                const uint32_t d = tq[(head + lane) & (WQ_TASKS - 1)];
                const int slot = (int)(d >> 10);
                const int64_t oi = ouser[slot];
                sweep_task<MAXM, C>(P, kinfo, orow + slot * MAXM, obeat + slot * MAXM, oi,
                                    P.uoff0 + oi * (int64_t)(M * C), (int)(d & 31u), (int)((d >> 5) & 31u), sink);
            }
            __syncwarp();
        };
        for (int64_t base = (int64_t)blockIdx.x * THREADS; base < P.N; base += (int64_t)gridDim.x * THREADS) {
            const int64_t i = base + threadIdx.x;
            const int64_t e0 = P.uoff0 + i * (int64_t)(M * C);
            uint32_t pd = 0u, shm = 0u;
            const unsigned wmask = __ballot_sync(0xffffffffu, i < P.N);  // lanes that run a user
            if (i < P.N)
                pd = csr_user_fast<MAXM, C, MODE>(P, S, i, e0, lamf, kinfo, rfix, dsum, psum, x_bits, sink,
                                                  nullptr, shm, wmask, orow, obeat, otail);
            // enqueue the user's pairs; its row was written to owner slot otail + rank
            const unsigned ob = __ballot_sync(0xffffffffu, pd != 0u);
            const int n = pair_count(pd);
            int x = n;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            const int total = __shfl_sync(0xffffffffu, x, 31);
            if (pd) {
                const unsigned slot = (otail + __popc(ob & lt)) & (WQ_OWN - 1);
                ouser[slot] = i;
                for (int t = 0; t < n; ++t)
                    tq[(tail + (unsigned)(x - n + t)) & (WQ_TASKS - 1)] =
                        (uint16_t)((slot << 10) | (unsigned)pair_first(pd, t) | ((unsigned)pair_second(pd, t) << 5));
            }
            tail += (unsigned)total;
            otail += (unsigned)__popc(ob);
            __syncwarp();
            while (tail - head >= 32u) {
                round(32);
                head += 32u;
            }
        }
        if (tail != head) round((int)(tail - head));
        return;
    }
    for (int64_t base = (int64_t)blockIdx.x * THREADS; base < P.N; base += (int64_t)gridDim.x * THREADS) {
        const int64_t i = base + threadIdx.x;
        const bool valid = i < P.N;
        int64_t e0;
        int nnz;
        if constexpr (C > 0) {
            nnz = M * C;
            e0 = P.uoff0 + i * (int64_t)nnz;
        } else {
            if (threadIdx.x == 0) s_base = P.uoff[base];
            nnz = 0;
            if (valid) {
                const uint8_t *nzr = P.innz + (size_t)i * M;
                for (int j = 0; j < M; ++j) nnz += nzr[j];
            }
            const int excl = block_excl_scan<THREADS>(nnz, s_scan);
            e0 = s_base + excl;
        }
        uint32_t pending = 0u, shm = 0u;
        const unsigned wmask = __ballot_sync(0xffffffffu, valid && nnz <= 32);  // lanes of the register path
        if (valid) {
            bool done = false;
            if constexpr (MAXM <= 16) {
                if (nnz <= 32) {
                    pending = csr_user_fast<MAXM, C, MODE>(P, S, i, e0, lamf, kinfo, rfix, dsum, psum, x_bits,
                                                           sink, rows + (size_t)threadIdx.x * MAXM, shm, wmask);
                    done = true;
                }
            }
            if (!done) {
                float ptl[MAXM], mgl[MAXM];
                csr_user<MAXM, MODE>(P, S, i, e0, nnz, lamf, ptl, mgl, rfix, dsum, psum, x_bits, sink);
            }
        }
        if constexpr (MODE != MODE_STATE && MAXM <= 16) {
            const int64_t ee[1] = {e0};
            const uint32_t pend[1] = {pending};
            block_sweeps<MAXM, C, THREADS, 1>(P, kinfo, rows, base, ee, pend, sink);
        }
        if constexpr (C == 0) __syncthreads();
    }
}

template <int MAXM, int C, int MODE, int THREADS>
__global__ void __launch_bounds__(THREADS, 1) csr_pass_kernel(Params P, Scratch S, const double *lam,
                                                              uint32_t *x_bits, int round, int sets) {
    extern __shared__ __align__(16) unsigned char smem[];
    if (MODE == MODE_REFINE && S.ctr->n_unres[round] == 0) return;
    if (MODE != MODE_STATE && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&S.ctr->stats[0], 1ull);
    const SmemLayout L = smem_layout(KP_B_CSR, P.K, P.M, MAXM, THREADS, 0, MODE, sets);
    init_block_state<MODE>(P, S, lam, L, smem, round, blockIdx.x == 0);
    __syncthreads();
    unsigned long long dsum = 0ull, psum = 0ull;
    if (MODE == MODE_HIST) {
        WindowSink ws = make_window_sink(P, S, L, smem);
        csr_loop<MAXM, C, MODE, THREADS>(P, S, smem, L, x_bits, ws, dsum, psum, sets);
    } else if (MODE == MODE_REFINE) {
        RefineSink rs = make_refine_sink(P, S, L, smem);
        csr_loop<MAXM, C, MODE, THREADS>(P, S, smem, L, x_bits, rs, dsum, psum, sets);
    } else {
        NullSink ns;
        csr_loop<MAXM, C, MODE, THREADS>(P, S, smem, L, x_bits, ns, dsum, psum, sets);
    }
    flush_block_state<MODE>(P, S, L, smem, dsum, psum, -1, MODE == MODE_HIST && C > 0);
}

// Knapsacks that three or more items of one user use (listed at creation; a
// few per cent of the shared ones): one thread per (user, knapsack), the
// user's reduced costs recomputed in the same order as the user pass, and
// Algorithm 4's Map by the exchange form of the sweep (kinetic beyond XMAX
// moving lines).  Keeping them out of the user pass keeps its sweep phase
// uniform across the lanes.  The blocks own buffer blocks
// [rare_blk0, rare_blk0 + rare_grid).
constexpr int RARE_THREADS = 512;
constexpr int XMAX = 3;

template <int MAXM, int C, class Sink>
__device__ __forceinline__ void rare_task(const Params &P, const float4 *kinfo, int64_t i, int e,
                                          Sink &sink) {
    const int M = P.M;
    const Tree &T = P.tree;
    const int64_t e0 = C > 0 ? P.uoff0 + i * (int64_t)(M * C) : P.uoff[i];
    const uint8_t *nzr = P.innz + (size_t)i * M;
    const float *val = P.val + e0;
    const int16_t *kid = P.kidx + e0;
    const int k = kid[e];
    if constexpr (C > 0 && MAXM <= 16) {
        // registers: reduced costs, rank masks, the moving lines of k
        float w[MAXM];
        int it[XMAX] = {0, 0, 0};
        float sl[XMAX] = {0.f, 0.f, 0.f};
        int nj = 0;
        uint32_t J = 0u, pos = 0u;
#pragma unroll
        for (int j = 0; j < MAXM; ++j) {
            float acc = j < M ? __ldg(P.p + (size_t)i * M + j) : 0.f;
#pragma unroll
            for (int q = 0; q < C; ++q) {
                const int f = j * C + q;
                const float v = j < M ? __ldg(val + f) : 0.f;
                const int kk = j < M ? (int)kid[f] : 0;
                acc = fmaf(-kinfo[kk].x, v, acc);
                if (j < M && kk == k && v > 0.f) {
#pragma unroll
                    for (int s2 = 0; s2 < XMAX; ++s2)
                        if (s2 == nj) {
                            it[s2] = j;
                            sl[s2] = v;
                        }
                    ++nj;
                    J |= 1u << j;
                }
            }
            w[j] = acc;
            if (j < M && acc > 0.f) pos |= 1u << j;
        }
        uint32_t bt[MAXM];
#pragma unroll
        for (int j = 0; j < MAXM; ++j) bt[j] = 0u;
#pragma unroll
        for (int j = 1; j < MAXM; ++j)
#pragma unroll
            for (int j2 = 0; j2 < j; ++j2) {
                const bool first = w[j2] >= w[j];  // j2 < j wins ties
                bt[j] |= first ? (1u << j2) : 0u;
                bt[j2] |= first ? 0u : (1u << j);
            }
        uint32_t SF = pos & ~J;  // Algorithm 1 over the fixed lines
        for (int l = 0; l < T.L; ++l) {
            const uint32_t inl = SF & (uint32_t)T.items[l];
            const int cap = T.cap[l];
            uint32_t drop = 0u;
#pragma unroll
            for (int j = 0; j < MAXM; ++j)
                if (((inl >> j) & 1u) && __popc(bt[j] & inl) >= cap) drop |= 1u << j;
            SF &= ~drop;
        }
        // every event lies at or below a moving line's zero crossing: nothing
        // to emit when all of them lie below the pass's floor (low_bound)
        const float tk = kinfo[k].w;
        bool any = false;
#pragma unroll
        for (int q = 0; q < XMAX; ++q) any |= q < nj && pick(w, it[q]) >= tk * sl[q];
        if (nj <= XMAX && !any) return;
        if (nj <= XMAX) {
            exchange_sweep<XMAX, MAXM>(w, SF, nj, it, sl, kinfo[k].x, T, k, sink);
            return;
        }
    }
    // general rows, or more than XMAX moving lines: the kinetic sweep
    float pt[KP_MAX_M], sv[KP_MAX_M];
    uint64_t Jm = 0;
    int f = 0;
    for (int j = 0; j < M; ++j) {
        float acc = __ldg(P.p + (size_t)i * M + j);
        sv[j] = 0.f;
        const int c = C > 0 ? C : (int)nzr[j];
        for (int q = 0; q < c; ++q, ++f) {
            const float v = __ldg(val + f);
            const int kk = kid[f];
            acc = fmaf(-kinfo[kk].x, v, acc);
            if (kk == k && v > 0.f) {
                sv[j] = v;
                Jm |= 1ull << j;
            }
        }
        pt[j] = acc;
    }
    sweep_k<KP_MAX_M>(pt, 1, sv, 1, M, Jm, kinfo[k].x, T, k, sink);
}

template <int MAXM, int C, int MODE>
__global__ void __launch_bounds__(RARE_THREADS, 2) rare_kernel(Params P, Scratch S, const double *lam, int round) {
    extern __shared__ __align__(16) unsigned char smem[];
    if (MODE == MODE_REFINE && S.ctr->n_unres[round] == 0) return;
    const SmemLayout L = smem_layout(KP_B_CSR, P.K, P.M, 1, RARE_THREADS, 0, MODE);
    init_block_state<MODE>(P, S, lam, L, smem, round, false);
    __syncthreads();
    const int blk = S.rare_blk0 + blockIdx.x;
    const float4 *kinfo = (const float4 *)(smem + L.kinfo);
    auto run = [&](auto &sink) {
        for (int64_t t = (int64_t)blockIdx.x * RARE_THREADS + threadIdx.x; t < S.nrare;
             t += (int64_t)gridDim.x * RARE_THREADS) {
            const unsigned long long rec = S.rare[t];
            rare_task<MAXM, C>(P, kinfo, (int64_t)(rec >> 5), (int)(rec & 31u), sink);
        }
    };
    if (MODE == MODE_HIST) {
        WindowSink ws = make_window_sink(P, S, L, smem);
        ws.blk = blk;
        run(ws);
    } else {
        RefineSink rs = make_refine_sink(P, S, L, smem);
        rs.blk = blk;
        run(rs);
    }
    flush_block_state<MODE>(P, S, L, smem, 0ull, 0ull, blk, MODE == MODE_HIST && C > 0);
}

// ------------------------------------------------------------------------------------------
// Dense layout: a tile of T users is staged in shared memory; reduced costs are
// computed per (user, item), the greedy per user, and consumption and the
// breakpoints per (user, knapsack).
// ------------------------------------------------------------------------------------------
// One tile of nu users starting at u0 (T users per tile): stage, reduce,
// Algorithm 1, then consumption and Algorithm 4's Map per (user, knapsack).
template <int MAXM, int MODE, int THREADS>
// staged: the tile's p and b are already in shared memory at tp_s / tb_s
// (the double-buffered pass; the caller synchronised the block after them);
// otherwise they are loaded here into the layout's single stage buffers.
__device__ __forceinline__ void dense_tile(const Params &P, const Scratch &S, const SmemLayout &L,
                                           unsigned char *smem, int64_t u0, int nu, int T,
                                           uint32_t *x_bits, unsigned long long &dsum,
                                           unsigned long long &psum, float *tp_s = nullptr,
                                           float *tb_s = nullptr) {
    const int M = P.M, K = P.K;
    const float *lamf = (const float *)(smem + L.lamf);
    const SFix rfix{(uint32_t *)(smem + L.rfix), K};
    const bool staged = tb_s != nullptr;
    float *tp = staged ? tp_s : (float *)(smem + L.tile_p);
    float *tb = staged ? tb_s : (float *)(smem + L.tile_b);
    float *pt = (float *)(smem + L.rows);
    uint64_t *selm = (uint64_t *)(smem + L.selm);
    const bool b_al = ((reinterpret_cast<uintptr_t>(P.b) & 15u) == 0) && ((M * K) % 4 == 0 || T % 4 == 0);
    const bool p_al = ((reinterpret_cast<uintptr_t>(P.p) & 15u) == 0) && ((M % 4) == 0 || T % 4 == 0);
    // stage the tile
    if (!staged) {
        const size_t nb = (size_t)nu * M * K;
        const float *src = P.b + (size_t)u0 * M * K;
        if (b_al) {
            const size_t n4 = nb >> 2;
            const float4 *s4 = reinterpret_cast<const float4 *>(src);
            float4 *d4 = reinterpret_cast<float4 *>(tb);
            for (size_t q = threadIdx.x; q < n4; q += THREADS) d4[q] = __ldg(s4 + q);
            for (size_t q = (n4 << 2) + threadIdx.x; q < nb; q += THREADS) tb[q] = __ldg(src + q);
        } else {
            for (size_t q = threadIdx.x; q < nb; q += THREADS) tb[q] = __ldg(src + q);
        }
        const size_t npn = (size_t)nu * M;
        const float *ps = P.p + (size_t)u0 * M;
        if (p_al) {
            const size_t n4 = npn >> 2;
            const float4 *s4 = reinterpret_cast<const float4 *>(ps);
            float4 *d4 = reinterpret_cast<float4 *>(tp);
            for (size_t q = threadIdx.x; q < n4; q += THREADS) d4[q] = __ldg(s4 + q);
            for (size_t q = (n4 << 2) + threadIdx.x; q < npn; q += THREADS) tp[q] = __ldg(ps + q);
        } else {
            for (size_t q = threadIdx.x; q < npn; q += THREADS) tp[q] = __ldg(ps + q);
        }
    }
    if (!staged) __syncthreads();
    // Sec. 4.2 reduced costs, four partial sums per item
    for (int idx = threadIdx.x; idx < nu * M; idx += THREADS) {
        const float *br = tb + (size_t)idx * K;
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        int k = 0;
        for (; k + 3 < K; k += 4) {
            a0 = fmaf(lamf[k], br[k], a0);
            a1 = fmaf(lamf[k + 1], br[k + 1], a1);
            a2 = fmaf(lamf[k + 2], br[k + 2], a2);
            a3 = fmaf(lamf[k + 3], br[k + 3], a3);
        }
        for (; k < K; ++k) a0 = fmaf(lamf[k], br[k], a0);
        pt[idx] = tp[idx] - ((a0 + a1) + (a2 + a3));
    }
    __syncthreads();
    // Algorithm 1 per user
    for (int u = threadIdx.x; u < nu; u += THREADS) {
        const float *ptu = pt + (size_t)u * M;
        uint64_t pos = 0;
        for (int j = 0; j < M; ++j)
            if (ptu[j] > 0.f) pos |= 1ull << j;
        Walk w;
        greedy_walk(ptu, 1, pos, P.tree, w);
        selm[u] = w.sel;
        if (MODE != MODE_REFINE) {
            const int64_t i = u0 + u;
            if (x_bits)
                for (int q = 0; q < P.W; ++q) x_bits[(size_t)i * P.W + q] = (uint32_t)(w.sel >> (32 * q));
            uint64_t r = w.sel;
            float du = 0.f, pu = 0.f;
            while (r) {
                int j = __ffsll((long long)r) - 1;
                r &= r - 1;
                du += ptu[j];
                pu += tp[(size_t)u * M + j];
            }
            dsum += fixmass(du, P.fixo);
            psum += fixmass(pu, P.fixo);
        }
    }
    __syncthreads();
    // per (user, knapsack): consumption and Algorithm 4's Map; thread t takes
    // the tasks t, t + THREADS, ... of the tile (task = u K + k, stepped without
    // division)
    const int du = THREADS / K, dk = THREADS - du * K;
    int u = threadIdx.x / K, k = threadIdx.x - u * K;
    const float4 *kinfo = (const float4 *)(smem + L.kinfo);
    const unsigned lane = threadIdx.x & 31u;
    uint32_t *dq = (uint32_t *)(smem + L.dq) + (threadIdx.x >> 5) * DQ_TASKS;
    int qh = 0, qn = 0;  // the warp's ring: head, count
    // the full sweep of a queued task (task = u K + k), its lines found again
    // from the tile exactly as in the first visit
    auto slow_task = [&](uint32_t task) {
        const int su = (int)(task / (uint32_t)K), sk = (int)(task - (uint32_t)su * (uint32_t)K);
        const float *bc = tb + (size_t)su * M * K + sk;
        const float *pu = pt + (size_t)su * M;
        const float lk = lamf[sk];
        const float t = kinfo[sk].w;
        int it[MAXM];
        float sl[MAXM];
        int n = 0;
        uint64_t fp = 0ull;
        for (int j = 0; j < M; ++j) {
            const float b = bc[(size_t)j * K];
            const float wj = pu[j];
            if (b > 0.f) {
                if (wj >= t * b) {
                    it[n] = j;
                    sl[n] = b;
                    ++n;
                }
            } else if (wj > 0.f) {
                fp |= 1ull << j;
            }
        }
        Walk wf;
        greedy_walk(pu, 1, fp, P.tree, wf);
        if (MODE == MODE_HIST) {
            WindowSink ws = make_window_sink(P, S, L, smem);
            live_sweep<MAXM>(pu, wf.sel, n, it, sl, lk, lk + t, P.tree, sk, ws);
        } else {
            RefineSink rs = make_refine_sink(P, S, L, smem);
            live_sweep<MAXM>(pu, wf.sel, n, it, sl, lk, lk + t, P.tree, sk, rs);
        }
    };
    // every lane takes the same number of rounds (the tasks' loops have
    // data-dependent trip counts: the warp meets again after each task)
    for (int base = 0; base < nu * K; base += THREADS, u += du, k += dk) {
        if (k >= K) {
            k -= K;
            ++u;
        }
        bool slow = false;
        int it[MAXM];     // the task's live lines (item, slope) and the
        float sl[MAXM];   // selection among its fixed lines, kept for a
        int nj = 0;       // sweep in place
        uint64_t sfsel = 0ull;
        if (u < nu) {
        const float *bcol = tb + (size_t)u * M * K + k;
        const float *ptu = pt + (size_t)u * M;
        const float lamk = lamf[k];
        const float tk = MODE == MODE_STATE ? 0.f : kinfo[k].w;
        // one pass over the items: lines positive at lambda_k = 0, live moving
        // lines (zero crossing can reach the pass's floor, see low_bound; the
        // others never enter at or above it), positive fixed lines
        uint64_t zpos = 0ull, livem = 0ull, fixedpos = 0ull;
        for (int j = 0; j < M; ++j) {
            const float b = bcol[(size_t)j * K];
            const float wj = ptu[j];
            if (fmaf(lamk, b, wj) > 0.f) zpos |= 1ull << j;
            if (b > 0.f) {
                if (wj >= tk * b) livem |= 1ull << j;
            } else if (wj > 0.f) {
                fixedpos |= 1ull << j;
            }
        }
        if (MODE != MODE_REFINE) {
            uint64_t r = selm[u];
            unsigned long long acc = 0ull;
            while (r) {
                int j = __ffsll((long long)r) - 1;
                r &= r - 1;
                acc += bmass(bcol[(size_t)j * K], P.bscale);
            }
            if (acc) rfix.add64(k, acc);
            if (MODE == MODE_HIST && tk < __int_as_float(0x7f800000)) {
                // the user's whole emitted mass, its k-consumption as lambda_k -> 0+
                // (Algorithm 1 at lambda_k = 0; at lambda_k^t = 0 the consumption
                // above): the selection reads it to decide lambda_k = 0, so the
                // sweep needs only the lines that reach the window
                unsigned long long tot = acc;
                if (lamk > 0.f) {
                    tot = 0ull;
                    if (zpos) {
                        float z[MAXM];
                        uint64_t q = zpos;
                        while (q) {
                            const int j = __ffsll((long long)q) - 1;
                            q &= q - 1;
                            z[j] = fmaf(lamk, bcol[(size_t)j * K], ptu[j]);
                        }
                        Walk w0;
                        greedy_walk(z, 1, zpos, P.tree, w0);
                        uint64_t r0 = w0.sel;
                        while (r0) {
                            const int j = __ffsll((long long)r0) - 1;
                            r0 &= r0 - 1;
                            tot += bmass(bcol[(size_t)j * K], P.bscale);
                        }
                    }
                }
                if (tot) SFix{(uint32_t *)(smem + L.reg3), 6 * K}.add64(4 * K + k, tot);  // bin (below, 0)
            }
        }
        if (MODE != MODE_STATE && livem) {
            uint64_t q = livem;
            while (q) {
                const int j = __ffsll((long long)q) - 1;
                q &= q - 1;
                it[nj] = j;
                sl[nj] = bcol[(size_t)j * K];
                ++nj;
            }
            Walk wf;
            greedy_walk(ptu, 1, fixedpos, P.tree, wf);  // selection among the fixed lines
            sfsel = wf.sel;
            if (MODE == MODE_HIST) {
                WindowSink ws = make_window_sink(P, S, L, smem);
                slow = !live_shortcut<MAXM>(ptu, sfsel, nj, it, sl, lamk, lamk + tk, P.tree, k, ws);
            } else {
                RefineSink rs = make_refine_sink(P, S, L, smem);
                slow = !live_shortcut<MAXM>(ptu, sfsel, nj, it, sl, lamk, lamk + tk, P.tree, k, rs);
            }
        }
        }
        if (MODE != MODE_STATE) {
            // tasks the shortcut did not settle: with most lanes of the round
            // among them the full sweep runs in place; otherwise they wait in
            // the warp's ring and 32 of them at a time run it on all lanes
            const unsigned bal = __ballot_sync(0xffffffffu, slow);
            if (__popc(bal) >= DQ_INPLACE) {
                if (slow) {
                    const float lk = lamf[k];
                    const float *pu = pt + (size_t)u * M;
                    if (MODE == MODE_HIST) {
                        WindowSink ws = make_window_sink(P, S, L, smem);
                        live_sweep<MAXM>(pu, sfsel, nj, it, sl, lk, lk + kinfo[k].w, P.tree, k, ws);
                    } else {
                        RefineSink rs = make_refine_sink(P, S, L, smem);
                        live_sweep<MAXM>(pu, sfsel, nj, it, sl, lk, lk + kinfo[k].w, P.tree, k, rs);
                    }
                }
            } else if (bal) {
                if (slow) dq[(qh + qn + __popc(bal & ((1u << lane) - 1u))) & (DQ_TASKS - 1)] = (uint32_t)(u * K + k);
                qn += __popc(bal);
                __syncwarp();
                if (qn >= 32) {
                    const uint32_t task = dq[(qh + (int)lane) & (DQ_TASKS - 1)];
                    qh = (qh + 32) & (DQ_TASKS - 1);
                    qn -= 32;
                    slow_task(task);
                }
            }
        }
        __syncwarp();
    }
    if (MODE != MODE_STATE && qn > 0) {
        if ((int)lane < qn) slow_task(dq[(qh + (int)lane) & (DQ_TASKS - 1)]);
        __syncwarp();
    }
    __syncthreads();
}

// Longest wait for a tile's bulk copies (ns): far above any copy's duration;
// reaching it sets KP_ETIMEOUT in the device status.
constexpr uint64_t STAGE_WAIT_NS = 2000000000ull;

// pipe = 1: the tiles are staged by bulk asynchronous copies into two
// buffers, the next tile's copy issued (by one thread) before the current
// tile is computed, completion counted on one mbarrier per buffer; needs p and
// b 16-byte aligned and T a multiple of 4 (every tile then starts on a 16-byte
// boundary; the bytes of a ragged last tile beyond a multiple of 16 are loaded
// directly).  pipe = 0: each tile is loaded synchronously, then computed.
template <int MAXM, int MODE, int THREADS>
__global__ void __launch_bounds__(THREADS, 2) dense_pass_kernel(Params Pk, Scratch S, const double *lam,
                                                             uint32_t *x_bits, int round, int T, int pipe) {
    extern __shared__ __align__(16) unsigned char smem[];
    if (MODE == MODE_REFINE && S.ctr->n_unres[round] == 0) return;
    if (MODE != MODE_STATE && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&S.ctr->stats[0], 1ull);
    // the parameters (the laminar family the sweeps index at run time among
    // them) are read from a shared copy: 4-5 % faster than from the kernel's
    // parameters on both dense workloads
    __shared__ Params P;
    if (threadIdx.x == 0) P = Pk;
    __syncthreads();
    const SmemLayout L = smem_layout(KP_B_DENSE, P.K, P.M, MAXM, THREADS, T, MODE, 1, pipe ? 2 : 1);
    init_block_state<MODE>(P, S, lam, L, smem, round, blockIdx.x == 0);
    __syncthreads();
    unsigned long long dsum = 0ull, psum = 0ull;
    const int64_t ntiles = (P.N + T - 1) / T;
    if (!pipe) {
        for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            const int64_t u0 = tile * T;
            const int nu = (int)((P.N - u0) < T ? (P.N - u0) : T);
            dense_tile<MAXM, MODE, THREADS>(P, S, L, smem, u0, nu, T, x_bits, dsum, psum);
        }
        flush_block_state<MODE>(P, S, L, smem, dsum, psum);
        return;
    }
    const int M = P.M, K = P.K;
    uint64_t *bar = (uint64_t *)(smem + L.bars);
    float *tpb[2] = {(float *)(smem + L.tile_p), (float *)(smem + L.tile_p2)};
    float *tbb[2] = {(float *)(smem + L.tile_b), (float *)(smem + L.tile_b2)};
    // bytes of a tile the bulk copies take (multiples of 16) and all its bytes
    auto tile_users = [&](int64_t tile) {
        const int64_t u0 = tile * T;
        return (int)((P.N - u0) < T ? (P.N - u0) : T);
    };
    auto issue = [&](int64_t tile, int buf) {  // one thread
        const int64_t u0 = tile * T;
        const int nu = tile_users(tile);
        const uint32_t bb = (uint32_t)(((size_t)nu * M * K * 4) & ~(size_t)15);
        const uint32_t bp = (uint32_t)(((size_t)nu * M * 4) & ~(size_t)15);
        fence_proxy_async_shared();
        mbar_arrive_expect_tx(&bar[buf], bb + bp);
        if (bb) bulk_copy_g2s(tbb[buf], P.b + (size_t)u0 * M * K, bb, &bar[buf]);
        if (bp) bulk_copy_g2s(tpb[buf], P.p + (size_t)u0 * M, bp, &bar[buf]);
    };
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init_fence();
    }
    __syncthreads();
    // thread 0's count, per buffer, of the copies issued and of the phases it saw complete
    uint32_t iss0 = 0u, iss1 = 0u, done0 = 0u, done1 = 0u;
    int64_t tile = blockIdx.x;
    if (tile < ntiles && threadIdx.x == 0) {
        issue(tile, 0);
        ++iss0;
    }
    bool ok = true;
    for (int n = 0; tile < ntiles; tile += gridDim.x, ++n) {
        const int cur = n & 1;
        const int64_t nxt = tile + gridDim.x;
        // the other buffer was last read by the previous tile, which every
        // thread finished (the barrier at the end of dense_tile)
        if (nxt < ntiles && threadIdx.x == 0) {
            issue(nxt, cur ^ 1);
            if (cur) ++iss0;
            else ++iss1;
        }
        const bool got = mbar_wait(&bar[cur], (uint32_t)((n >> 1) & 1), STAGE_WAIT_NS);
        if (threadIdx.x == 0 && got) {
            if (cur) ++done1;
            else ++done0;
        }
        ok = __syncthreads_and(got) != 0;
        if (!ok) break;
        const int64_t u0 = tile * T;
        const int nu = tile_users(tile);
        {  // the bytes past the last multiple of 16 (ragged last tile)
            const size_t nb = (size_t)nu * M * K, np = (size_t)nu * M;
            for (size_t q = ((nb * 4) & ~(size_t)15) / 4 + threadIdx.x; q < nb; q += THREADS)
                tbb[cur][q] = __ldg(P.b + (size_t)u0 * M * K + q);
            for (size_t q = ((np * 4) & ~(size_t)15) / 4 + threadIdx.x; q < np; q += THREADS)
                tpb[cur][q] = __ldg(P.p + (size_t)u0 * M + q);
        }
        __syncthreads();
        dense_tile<MAXM, MODE, THREADS>(P, S, L, smem, u0, nu, T, x_bits, dsum, psum, tpb[cur], tbb[cur]);
    }
    if (!ok) {
        // a copy did not complete in time: report it and wait (bounded) for
        // every copy still in flight, so that none lands after the block left
        if (threadIdx.x == 0) {
            atomicOr(&S.ctr->status, 1 << KP_ETIMEOUT);
            for (uint32_t w = done0; w < iss0; ++w) (void)mbar_wait(&bar[0], w & 1u, STAGE_WAIT_NS);
            for (uint32_t w = done1; w < iss1; ++w) (void)mbar_wait(&bar[1], w & 1u, STAGE_WAIT_NS);
        }
        __syncthreads();
        return;
    }
    flush_block_state<MODE>(P, S, L, smem, dsum, psum);
}

// Batched pass: one persistent launch over the tiles of many dense instances.
// Blocks take tiles from the pass's counter; consecutive tiles belong to the
// same instance, so a block switches instance rarely; at a switch it flushes
// the previous instance's block state into that instance's scratch and loads
// the next instance's parameters and multipliers.  Every sum is an integer
// sum, so the result does not depend on which block took which tile.
template <int MAXM, int MODE, int THREADS>
__global__ void __launch_bounds__(THREADS, 2) dense_batch_kernel(BatchDev B, const double *lam_all,
                                                              uint32_t *x_all, int round) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ Params sP;
    __shared__ Scratch sS;
    __shared__ int s_skip;
    __shared__ long long s_t[2];  // alternate slots: a thread still reading one never sees it rewritten
    int cur = -1;
    unsigned long long dsum = 0ull, psum = 0ull;
    SmemLayout L;
    // thread 0 claims the next tile while the block works on the current one,
    // so the counter's round trip is off the block's path
    long long nxt = 0;
    if (threadIdx.x == 0) nxt = (long long)atomicAdd(&B.next[round], 1ull);
    for (int it = 0;; ++it) {
        if (threadIdx.x == 0) s_t[it & 1] = nxt;
        __syncthreads();
        const int64_t t = s_t[it & 1];
        if (t >= B.ntiles) break;
        if (threadIdx.x == 0) nxt = (long long)atomicAdd(&B.next[round], 1ull);
        const int inst = B.tile_inst[t];
        if (inst != cur) {
            if (cur >= 0 && !s_skip) flush_block_state<MODE>(sP, sS, L, smem, dsum, psum);
            __syncthreads();
            if (threadIdx.x == 0) {
                sP = B.P[inst];
                sS = B.S[inst];
                s_skip = MODE == MODE_REFINE && sS.ctr->n_unres[round] == 0;
            }
            __syncthreads();
            cur = inst;
            dsum = psum = 0ull;
            L = smem_layout(KP_B_DENSE, sP.K, sP.M, MAXM, THREADS, sP.tile, MODE);
            if (!s_skip) init_block_state<MODE>(sP, sS, lam_all + B.koff[inst], L, smem, round, B.tile_u0[t] == 0);
            __syncthreads();
        }
        if (s_skip) continue;
        const int64_t u0 = B.tile_u0[t];
        const int nu = (int)((sP.N - u0) < sP.tile ? (sP.N - u0) : sP.tile);
        dense_tile<MAXM, MODE, THREADS>(sP, sS, L, smem, u0, nu, sP.tile,
                                        x_all ? x_all + B.xoff[inst] : nullptr, dsum, psum);
    }
    if (cur >= 0 && !s_skip) flush_block_state<MODE>(sP, sS, L, smem, dsum, psum);
}

int max_optin_smem() {
    static int v = 0;
    if (!v) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (v <= 0) v = 48 * 1024;
    }
    return v;
}

constexpr int CSR_THREADS = 512;
// the consumption pass (no breakpoints) of rows of up to 10 items needs fewer
// registers: 24 warps per SM instead of 16 hide more of its load latency
constexpr int CSR_STATE_THREADS = 768;
template <int MAXM, int MODE>
constexpr int csr_threads() { return MODE == MODE_STATE && MAXM <= 10 ? CSR_STATE_THREADS : CSR_THREADS; }
constexpr int DENSE_THREADS = 256;


template <class Kern>
cudaError_t prepare_kernel(Kern kern, int *max_dyn) {
    if (*max_dyn >= 0) return cudaSuccess;
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    const int md = max_optin_smem() - (int)fa.sharedSizeBytes;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, md);
    if (e != cudaSuccess) return e;
    *max_dyn = md;
    return cudaSuccess;
}

template <int MAXM, int C, int MODE>
cudaError_t launch_csr(const Params &P, const Scratch &S, const double *lam, uint32_t *x_bits,
                       int round, cudaStream_t st, int *occupancy_out) {
    constexpr int THR = csr_threads<MAXM, MODE>();
    auto kern = csr_pass_kernel<MAXM, C, MODE, THR>;
    static int max_dyn = -1;  // once per instantiation, before any stream capture
    cudaError_t e = prepare_kernel(kern, &max_dyn);
    if (e != cudaSuccess) return e;
    // regular rows: per-warp pair queues (sets = 0) when they fit next to the
    // per-knapsack state, else per-thread rows swept after every tile
    int sets = (C > 0 && MODE != MODE_STATE && MAXM <= 16) ? 0 : 1;
    SmemLayout L = smem_layout(KP_B_CSR, P.K, P.M, MAXM, THR, 0, MODE, sets);
    if (L.total > (size_t)max_dyn && sets != 1) {
        sets = 1;
        L = smem_layout(KP_B_CSR, P.K, P.M, MAXM, THR, 0, MODE, sets);
    }
    if (L.total > (size_t)max_dyn) return cudaErrorInvalidConfiguration;
    if (occupancy_out)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occupancy_out, kern, THR, L.total);
    kern<<<S.G, THR, L.total, st>>>(P, S, lam, x_bits, round, sets);
    return cudaGetLastError();
}

template <int MAXM, int MODE>
cudaError_t launch_dense(const Params &P, const Scratch &S, const double *lam, uint32_t *x_bits,
                         int round, cudaStream_t st, int *occupancy_out) {
    int T = P.tile > 0 ? P.tile : dense_tile_users(P);
    auto kern = dense_pass_kernel<MAXM, MODE, DENSE_THREADS>;
    static int max_dyn = -1;
    cudaError_t e = prepare_kernel(kern, &max_dyn);
    if (e != cudaSuccess) return e;
    // staging mode 1: double-buffered with half a tile per buffer (the two
    // buffers take the shared memory of one tile, so as many blocks fit on an
    // SM); needs 16-byte aligned p and b and a buffer of a multiple of 4 users
    int pipe = 0;
    SmemLayout L = smem_layout(KP_B_DENSE, P.K, P.M, MAXM, DENSE_THREADS, T, MODE);
    const int Th = (T / 2) & ~3;
    if (P.stage == 1 && Th >= 4 && (reinterpret_cast<uintptr_t>(P.b) & 15u) == 0 && (reinterpret_cast<uintptr_t>(P.p) & 15u) == 0) {
        const SmemLayout L2 = smem_layout(KP_B_DENSE, P.K, P.M, MAXM, DENSE_THREADS, Th, MODE, 1, 2);
        if (L2.total <= (size_t)max_dyn) {
            pipe = 1;
            T = Th;
            L = L2;
        }
    }
    if (L.total > (size_t)max_dyn) return cudaErrorInvalidConfiguration;
    if (occupancy_out)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occupancy_out, kern, DENSE_THREADS, L.total);
    kern<<<S.G, DENSE_THREADS, L.total, st>>>(P, S, lam, x_bits, round, T, pipe);
    return cudaGetLastError();
}

template <int MAXM, int MODE>
cudaError_t launch_t(const Params &P, const Scratch &S, const double *lam, uint32_t *x_bits,
                     int round, cudaStream_t st, int *occ) {
    if (P.layout != KP_B_CSR) return launch_dense<MAXM, MODE>(P, S, lam, x_bits, round, st, occ);
    if constexpr (MAXM <= 16) {
        if (P.creg == 1) return launch_csr<MAXM, 1, MODE>(P, S, lam, x_bits, round, st, occ);
        if (P.creg == 2) return launch_csr<MAXM, 2, MODE>(P, S, lam, x_bits, round, st, occ);
    }
    return launch_csr<MAXM, 0, MODE>(P, S, lam, x_bits, round, st, occ);
}

template <int MAXM>
cudaError_t launch_m(const Params &P, const Scratch &S, const double *lam, int mode, int round,
                     uint32_t *x_bits, cudaStream_t st, int *occ) {
    switch (mode) {
        case MODE_STATE: return launch_t<MAXM, MODE_STATE>(P, S, lam, x_bits, round, st, occ);
        case MODE_HIST: return launch_t<MAXM, MODE_HIST>(P, S, lam, x_bits, round, st, occ);
        default: return launch_t<MAXM, MODE_REFINE>(P, S, lam, x_bits, round, st, occ);
    }
}

cudaError_t dispatch(const Params &P, const Scratch &S, const double *lam, int mode, int round,
                     uint32_t *x_bits, cudaStream_t st, int *occ) {
    if (P.M <= 8) return launch_m<8>(P, S, lam, mode, round, x_bits, st, occ);
    if (P.M <= 10) return launch_m<10>(P, S, lam, mode, round, x_bits, st, occ);
    if (P.M <= 16) return launch_m<16>(P, S, lam, mode, round, x_bits, st, occ);
    return launch_m<64>(P, S, lam, mode, round, x_bits, st, occ);
}

template <int MAXM, int MODE>
cudaError_t launch_batch_t(const BatchDev &B, size_t smem, int grid, const double *lam, int round,
                           uint32_t *x_all, cudaStream_t st, int *occupancy_out) {
    auto kern = dense_batch_kernel<MAXM, MODE, DENSE_THREADS>;
    static int max_dyn = -1;
    cudaError_t e = prepare_kernel(kern, &max_dyn);
    if (e != cudaSuccess) return e;
    if (smem > (size_t)max_dyn) return cudaErrorInvalidConfiguration;
    if (occupancy_out)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occupancy_out, kern, DENSE_THREADS, smem);
    kern<<<grid, DENSE_THREADS, smem, st>>>(B, lam, x_all, round);
    return cudaGetLastError();
}

template <int MAXM>
cudaError_t launch_batch_m(const BatchDev &B, size_t smem, int grid, const double *lam, int mode,
                           int round, uint32_t *x_all, cudaStream_t st, int *occ) {
    switch (mode) {
        case MODE_STATE: return launch_batch_t<MAXM, MODE_STATE>(B, smem, grid, lam, round, x_all, st, occ);
        case MODE_HIST: return launch_batch_t<MAXM, MODE_HIST>(B, smem, grid, lam, round, x_all, st, occ);
        default: return launch_batch_t<MAXM, MODE_REFINE>(B, smem, grid, lam, round, x_all, st, occ);
    }
}

cudaError_t batch_dispatch(const BatchDev &B, int maxm, size_t smem, int grid, const double *lam, int mode,
                           int round, uint32_t *x_all, cudaStream_t st, int *occ) {
    if (maxm <= 8) return launch_batch_m<8>(B, smem, grid, lam, mode, round, x_all, st, occ);
    if (maxm <= 10) return launch_batch_m<10>(B, smem, grid, lam, mode, round, x_all, st, occ);
    if (maxm <= 16) return launch_batch_m<16>(B, smem, grid, lam, mode, round, x_all, st, occ);
    return launch_batch_m<64>(B, smem, grid, lam, mode, round, x_all, st, occ);
}

}  // namespace

// Users per shared-memory tile of the dense pass: a 64 KB tile of b, and at
// most 96 KB for everything staged per user (b, p, p~ and the selection), so
// that two blocks fit on an SM also when K is small and M large.
int dense_tile_users(const Params &P) {
    long long per = (long long)P.M * P.K * 4;
    long long T = DENSE_TILE_BYTES / per;
    const long long T2 = DENSE_USER_BYTES / (per + 8LL * P.M + 8);
    if (T2 < T) T = T2;
    if (T > 256) T = 256;
    if (T >= 4) T &= ~3LL;
    if (T < 1) T = 1;
    return (int)T;
}

size_t dense_smem_bytes(const Params &P, int mode) {
    return smem_layout(KP_B_DENSE, P.K, P.M, 64, DENSE_THREADS, P.tile ? P.tile : dense_tile_users(P), mode).total;
}

cudaError_t launch_batch_pass(const BatchDev &B, int maxm, size_t smem, int grid, const double *lam,
                              int mode, int round, uint32_t *x_all, cudaStream_t st) {
    return batch_dispatch(B, maxm, smem, grid, lam, mode, round, x_all, st, nullptr);
}

// Persistent grid of the batched pass: SM count x resident blocks of the histogram mode.
int batch_grid_size(int maxm, size_t smem) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    BatchDev dummy{};
    int occ = 0;
    for (int mode = 0; mode < 3; ++mode) {
        int o = 0;
        if (batch_dispatch(dummy, maxm, smem, 1, nullptr, mode, 0, nullptr, 0, &o) != cudaSuccess || o < 1) {
            (void)cudaGetLastError();
            return 0;
        }
        occ = mode == 0 ? o : (o < occ ? o : occ);
    }
    if (occ > 4) occ = 4;
    return sms * occ;
}

template <int MAXM, int C, int MODE>
cudaError_t launch_rare_t(const Params &P, const Scratch &S, const double *lam, int round, cudaStream_t st,
                          bool prepare_only) {
    auto kern = rare_kernel<MAXM, C, MODE>;
    static int max_dyn = -1;  // once per instantiation, before any stream capture
    cudaError_t e = prepare_kernel(kern, &max_dyn);
    if (e != cudaSuccess || prepare_only) return e;
    const SmemLayout L = smem_layout(KP_B_CSR, P.K, P.M, 1, RARE_THREADS, 0, MODE);
    if (L.total > (size_t)max_dyn) return cudaErrorInvalidConfiguration;
    kern<<<S.rare_grid, RARE_THREADS, L.total, st>>>(P, S, lam, round);
    return cudaGetLastError();
}

template <int MODE>
cudaError_t launch_rare(const Params &P, const Scratch &S, const double *lam, int round, cudaStream_t st,
                        bool prepare_only) {
    if (P.creg == 2 || P.creg == 1) {
        const bool two = P.creg == 2;
        if (P.M <= 8) return two ? launch_rare_t<8, 2, MODE>(P, S, lam, round, st, prepare_only)
                                 : launch_rare_t<8, 1, MODE>(P, S, lam, round, st, prepare_only);
        if (P.M <= 10) return two ? launch_rare_t<10, 2, MODE>(P, S, lam, round, st, prepare_only)
                                  : launch_rare_t<10, 1, MODE>(P, S, lam, round, st, prepare_only);
        if (P.M <= 16) return two ? launch_rare_t<16, 2, MODE>(P, S, lam, round, st, prepare_only)
                                  : launch_rare_t<16, 1, MODE>(P, S, lam, round, st, prepare_only);
    }
    return launch_rare_t<64, 0, MODE>(P, S, lam, round, st, prepare_only);
}

cudaError_t launch_user_pass(const Params &P, const Scratch &S, const double *lambda, int mode,
                             int round, uint32_t *x_bits, cudaStream_t st) {
    cudaError_t e = dispatch(P, S, lambda, mode, round, x_bits, st, nullptr);
    if (e != cudaSuccess || mode == MODE_STATE || S.nrare == 0 || S.rare_grid == 0) return e;
    return mode == MODE_HIST ? launch_rare<MODE_HIST>(P, S, lambda, round, st, false)
                             : launch_rare<MODE_REFINE>(P, S, lambda, round, st, false);
}

// Persistent grid: SM count x resident blocks of the heaviest mode.
int pass_grid_size(const Params &P) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int occ = 0;
    Scratch dummy{};
    if (dispatch(P, dummy, nullptr, MODE_HIST, 0, nullptr, 0, &occ) != cudaSuccess || occ < 1) occ = 1;
    int occ2 = 0;
    if (dispatch(P, dummy, nullptr, MODE_REFINE, 0, nullptr, 0, &occ2) == cudaSuccess && occ2 >= 1 &&
        occ2 < occ)
        occ = occ2;
    int occ3 = 0;
    if (dispatch(P, dummy, nullptr, MODE_STATE, 0, nullptr, 0, &occ3) == cudaSuccess && occ3 >= 1 &&
        occ3 < occ)
        occ = occ3;
    if (P.layout == KP_B_CSR) {  // kernel attributes of the rare-knapsack sweeps
        launch_rare<MODE_HIST>(P, dummy, nullptr, 0, 0, true);
        launch_rare<MODE_REFINE>(P, dummy, nullptr, 0, 0, true);
    }
    (void)cudaGetLastError();  // the queries above report failures through their return values
    if (occ > 4) occ = 4;
    return sms * occ;
}

size_t pass_smem_bytes(const Params &P, int mode) {
    int maxm = P.M <= 8 ? 8 : (P.M <= 10 ? 10 : (P.M <= 16 ? 16 : 64));
    if (P.layout == KP_B_CSR)
        return smem_layout(KP_B_CSR, P.K, P.M, maxm, mode == MODE_STATE && maxm <= 10 ? CSR_STATE_THREADS : CSR_THREADS,
                           0, mode)
            .total;
    return smem_layout(KP_B_DENSE, P.K, P.M, maxm, DENSE_THREADS, dense_tile_users(P), mode).total;
}

namespace {

// One mbarrier that nothing arrives on: the staging pass's bounded wait runs
// out after limit_ns and the kernel reports it as the passes do.
__global__ void wait_selftest_kernel(uint64_t limit_ns, int32_t *status) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_init_fence();
    }
    __syncthreads();
    const bool got = mbar_wait(&bar, 0u, limit_ns);
    if (threadIdx.x == 0 && !got) atomicOr(status, 1 << KP_ETIMEOUT);
}

}  // namespace

cudaError_t launch_wait_selftest(uint64_t limit_ns, int32_t *status, cudaStream_t st) {
    wait_selftest_kernel<<<1, 32, 0, st>>>(limit_ns, status);
    return cudaGetLastError();
}

}  // namespace kp
