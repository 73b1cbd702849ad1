// kp_select.cu -- the small kernels around the user pass:
//   finalize_kernel  ordered FP64 sums of the per-block partials, R_k from
//                    the fixed-point accumulators, the dual objective
//                    (Eq. (5)) and the dual-descent update (Eq. (14)).
//   select_kernel    the Reduce of Algorithm 4 for every knapsack: find the
//                    breakpoint at which the mass accumulated from the top
//                    first exceeds B_k, from the exact masses above / inside /
//                    below the window and then exactly among the buffered
//                    breakpoints (radix selection on the FP32 bit patterns,
//                    8 bits per round), or by re-run passes with 256-way
//                    sub-histograms when the crossing is outside the window.
//   backward_kernel  Danskin gradient of the dual function.
//   validate_kernel  checks of Sec. 2's data assumptions at creation.
#include <cfloat>
#include <cstdint>

#include "kp_device.cuh"
#include "kp_internal.h"

namespace kp {

namespace {

__device__ __forceinline__ int bitlen32(uint32_t x) { return x ? 32 - __clz(x) : 0; }

// Largest half-width of the window, in keys (2^21 keys: about +-25 % in value).
// After a large move of lambda_k a window as wide as the miss holds more
// breakpoints than the buffer keeps, which costs re-run passes just as a miss
// does; on the 1e8-user workload the cap saves three passes of the first steps.
constexpr int WMAX_BITS = 21;

__device__ __forceinline__ unsigned long long budget_fixed(double Bk, int fixs) {
    double v = ldexp(Bk, fixs);
    if (!(v > 0.0)) return 0ull;
    if (v >= 1.8e19) return ~0ull;
    return (unsigned long long)floor(v);
}

__device__ __forceinline__ void finalize_body(const Params &P, const Scratch &S, const double *lam,
                                              double *R, double *dual, double *primal, double *g,
                                              double alpha, double *lam_next, int do_dd) {
    const int K = P.K;
    if (threadIdx.x == 0) {
        const double io = ldexp(1.0, -P.fixo);
        unsigned long long o0 = S.objfix[0], o1 = S.objfix[1];
        for (int q = 0; q < S.npeers; ++q) {  // the other shards' users
            o0 += S.peers[q].objfix[0];
            o1 += S.peers[q].objfix[1];
            S.peers[q].objfix[0] = 0ull;
            S.peers[q].objfix[1] = 0ull;
        }
        const double a = (double)o0 * io, b = (double)o1 * io;
        S.objfix[0] = 0ull;
        S.objfix[1] = 0ull;
        if (dual) *dual = a;
        if (primal) *primal = b;
        if (g) {
            double lb = 0.0;
            for (int k = 0; k < K; ++k) lb += lam[k] * P.B[k];
            *g = a + lb;
        }
    }
    __syncthreads();
    const double inv = ldexp(1.0, -P.fixs);
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        unsigned long long rf = S.Rfix[k];
        for (int q = 0; q < S.npeers; ++q) {
            rf += S.peers[q].Rfix[k];
            S.peers[q].Rfix[k] = 0ull;
        }
        const double Rk = (double)rf * inv;
        S.Rfix[k] = 0ull;
        if (R) R[k] = Rk;
        if (do_dd) {
            const double v = lam[k] + alpha * (Rk - P.B[k]);
            lam_next[k] = v > 0.0 ? v : 0.0;
        }
    }
}

__global__ void finalize_kernel(Params P, Scratch S, const double *lam, double *R, double *dual,
                                double *primal, double *g, double alpha, double *lam_next,
                                int do_dd) {
    finalize_body(P, S, lam, R, dual, primal, g, alpha, lam_next, do_dd);
}

// one block per instance of a batch; outputs (if given) at the instance's offsets
__global__ void batch_finalize_kernel(BatchDev B, const double *lam, double *R, double *dual,
                                      double *primal, double alpha, double *lam_next, int do_dd) {
    __shared__ Params sP;
    __shared__ Scratch sS;
    const int i = blockIdx.x;
    if (B.solo[i]) return;  // finalized by its own launch
    if (threadIdx.x == 0) {
        sP = B.P[i];
        sS = B.S[i];
    }
    __syncthreads();
    const int64_t ko = B.koff[i];
    finalize_body(sP, sS, lam + ko, R ? R + ko : nullptr, dual ? dual + i : nullptr,
                  primal ? primal + i : nullptr, nullptr, alpha, lam_next ? lam_next + ko : nullptr, do_dd);
}

// exact selection among the buffered breakpoints of knapsack k with key in
// [lo, hi): the key at which the mass accumulated from the top first exceeds
// `need`.  Block-wide; returns the key to every thread.
__device__ uint32_t exact_select(const Scratch &S, const Params &P, int k, uint32_t lo, uint32_t hi,
                                 unsigned long long need, bool *ok) {
    __shared__ unsigned long long h[NSUB];
    __shared__ uint32_t s_lo, s_w;
    __shared__ unsigned long long s_need;
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        s_lo = lo;
        s_w = hi - lo;
        s_need = need;
        s_ok = 1;
    }
    __syncthreads();
    for (int guard = 0; guard < 8; ++guard) {
        const uint32_t clo = s_lo, width = s_w;
        if (width <= 1) break;
        int sh = bitlen32(width - 1) - 8;
        if (sh < 0) sh = 0;
        const int nd = (int)(((width - 1) >> sh) + 1);
        for (int d = threadIdx.x; d < NSUB; d += blockDim.x) h[d] = 0ull;
        __syncthreads();
        for (int q = -1; q < S.npeers; ++q) {  // this shard's buffer, then the other shards'
            const Scratch &T = q < 0 ? S : S.peers[q];
            for (int gblk = 0; gblk < T.gspan; ++gblk) {
                const uint32_t cnt = T.bufcnt[(size_t)k * T.gspan + gblk];
                const uint2 *base = T.buf + ((size_t)k * T.gspan + gblk) * T.cap_kb;
                for (uint32_t s = threadIdx.x; s < cnt; s += blockDim.x) {
                    const uint2 e = base[s];
                    const uint32_t off = e.x - clo;
                    if (e.x >= clo && off < width)
                        atomicAdd(&h[off >> sh], (unsigned long long)bmass(__uint_as_float(e.y), P.bscale));
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long acc = 0ull;
            int pick = -1;
            for (int d = nd - 1; d >= 0; --d) {
                if (acc + h[d] > s_need) {
                    pick = d;
                    break;
                }
                acc += h[d];
            }
            if (pick < 0) {  // inconsistent masses: cannot happen with a complete buffer
                s_ok = 0;
                pick = 0;
                acc = 0;
            }
            s_need -= acc;
            const uint32_t nlo = clo + ((uint32_t)pick << sh);
            const uint32_t span = sh == 0 ? 1u : (1u << sh);
            const uint32_t end = clo + width;
            s_lo = nlo;
            s_w = (end - nlo) < span ? (end - nlo) : span;
        }
        __syncthreads();
    }
    __syncthreads();
    *ok = s_ok != 0;
    return s_lo;
}

// Record lambda_k^{t+1} and choose the centre and window of the next pass.
// In the damped two-cycles that synchronous coordinate descent shows, the
// next value is closer to the value two steps back than to the last one, so
// when the last two moves alternate in sign the centre is lambda_k^t.  The
// half-width is twice the error of this pass's centre.
__device__ __forceinline__ void resolved(SelK &sk, int k, uint32_t key, float lam_t,
                                         double *lam_next) {
    lam_next[k] = key ? (double)__uint_as_float(key) : 0.0;
    const uint32_t cur = lam_t > 0.f ? __float_as_uint(lam_t) : 0u;
    const uint32_t prev = sk.prev_key;
    const bool osc = (key > cur && cur < prev) || (key < cur && cur > prev);
    uint32_t pred = osc ? cur : key;
    if (pred == 0u) pred = key ? key : (cur ? cur : sk.last_nz_key);
    if (key) {
        const uint32_t err = key > sk.ckey ? key - sk.ckey : sk.ckey - key;
        const int w = bitlen32(err) + 1;
        sk.w = w < WMIN_BITS ? WMIN_BITS : (w > WMAX_BITS ? WMAX_BITS : w);
        sk.last_nz_key = key;
    }
    sk.prev_key = cur;
    sk.for_key = key;
    sk.pred_key = pred;
    sk.state = 0;
}

__device__ __forceinline__ void unresolved(Scratch &S, SelK &sk, uint32_t lo, uint32_t hi,
                                           unsigned long long above, int round) {
    sk.state = 1;
    sk.lo = lo;
    sk.hi = hi;
    sk.above = above;
    atomicAdd(&S.ctr->n_unres[round + 1], 1);
}

__device__ __forceinline__ void select_body(const Params &P, Scratch &S, int k, const double *lam,
                                            double *lam_next, int round) {
    __shared__ SelK sk;
    __shared__ unsigned long long row[NSUB];
    __shared__ int s_pick;
    __shared__ unsigned long long s_above;
    if (S.block && !S.block[k]) {  // outside the block of a block coordinate-descent step
        if (round == 0 && threadIdx.x == 0) {
            lam_next[k] = lam[k];
            S.reg3[3 * k] = 0ull;
            S.reg3[3 * k + 1] = 0ull;
            S.reg3[3 * k + 2] = 0ull;
            S.ovf[k] = 0u;
        }
        return;
    }
    if (threadIdx.x == 0) sk = S.sel[k];
    __syncthreads();
    if (round > 0 && sk.state != 1) return;
    const unsigned long long Bfix = budget_fixed(P.B[k], P.fixs);
    const float lam_t = (float)lam[k];
    uint32_t ovf = S.ovf[k];
    for (int q = 0; q < S.npeers; ++q) ovf |= S.peers[q].ovf[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        S.ovf[k] = 0u;
        for (int q = 0; q < S.npeers; ++q) S.peers[q].ovf[k] = 0u;
        if (ovf) atomicAdd(&S.ctr->stats[2], 1ull);
    }
    if (round == 0) {
        // masses at/above, inside and below the window [wlo, whi), summed over the shards
        unsigned long long A = S.reg3[3 * k], W = S.reg3[3 * k + 1], Bl = S.reg3[3 * k + 2];
        for (int q = 0; q < S.npeers; ++q) {
            A += S.peers[q].reg3[3 * k];
            W += S.peers[q].reg3[3 * k + 1];
            Bl += S.peers[q].reg3[3 * k + 2];
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            S.reg3[3 * k] = 0ull;
            S.reg3[3 * k + 1] = 0ull;
            S.reg3[3 * k + 2] = 0ull;
            for (int q = 0; q < S.npeers; ++q) {
                S.peers[q].reg3[3 * k] = 0ull;
                S.peers[q].reg3[3 * k + 1] = 0ull;
                S.peers[q].reg3[3 * k + 2] = 0ull;
            }
        }
        // dense rows: Bl is the total mass (every user's consumption as
        // lambda_k -> 0+).  Regular CSR rows leave out of Bl the breakpoints
        // below both the window and lambda_k^t: the total is then known only
        // when there are none (lambda_k^t = 0, every breakpoint lies above it).
        const bool dense = P.layout == KP_B_DENSE;
        const bool skips_low = P.layout == KP_B_CSR && P.creg > 0 && P.M <= 16;
        const bool below_known = dense || !skips_low || !(lam_t > 0.f);
        const unsigned long long total = dense ? Bl : A + W + Bl;
        if (below_known && total <= Bfix) {  // the whole mass fits: lambda_k = 0
            if (threadIdx.x == 0) {
                resolved(sk, k, 0u, lam_t, lam_next);
                atomicAdd(&S.ctr->stats[1], 1ull);
                S.sel[k] = sk;
            }
            return;
        }
        if (A > Bfix) {  // crossing at or above the window
            if (threadIdx.x == 0) {
                unresolved(S, sk, sk.whi, KEY_INF, 0ull, round);
                S.sel[k] = sk;
            }
            return;
        }
        if (A + W > Bfix) {  // crossing inside the window
            if (!ovf) {
                bool ok = true;
                const uint32_t key = exact_select(S, P, k, sk.wlo, sk.whi, Bfix - A, &ok);
                if (threadIdx.x == 0) {
                    if (!ok) atomicOr(&S.ctr->status, 1 << KP_ESTATE);
                    resolved(sk, k, key, lam_t, lam_next);
                    S.sel[k] = sk;
                }
            } else if (threadIdx.x == 0) {
                unresolved(S, sk, sk.wlo, sk.whi, A, round);
                S.sel[k] = sk;
            }
            return;
        }
        if (threadIdx.x == 0) {  // crossing below the window
            unresolved(S, sk, 1u, sk.wlo > 1u ? sk.wlo : 2u, A + W, round);
            S.sel[k] = sk;
        }
        return;
    }

    // refine round: sub-histogram of [sk.lo, sk.hi)
    unsigned long long *grow = S.subhist + (size_t)k * NSUB;
    for (int q = threadIdx.x; q < NSUB; q += blockDim.x) {
        unsigned long long v = grow[q];
        grow[q] = 0ull;
        for (int r = 0; r < S.npeers; ++r) {  // the other shards' sub-histograms
            unsigned long long *pg = S.peers[r].subhist + (size_t)k * NSUB;
            v += pg[q];
            pg[q] = 0ull;
        }
        row[q] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int pick = -1;
        unsigned long long acc = sk.above;
        for (int b = NSUB - 1; b >= 0; --b) {
            if (acc + row[b] > Bfix) {
                pick = b;
                break;
            }
            acc += row[b];
        }
        s_pick = pick;
        s_above = acc;
    }
    __syncthreads();
    const int pick = s_pick;
    if (pick < 0) {
        if (threadIdx.x == 0) {
            if (sk.lo <= 1u) {  // the range reaches down to 0 and everything fits: lambda_k = 0
                resolved(sk, k, 0u, lam_t, lam_next);
                atomicAdd(&S.ctr->stats[1], 1ull);
            } else {  // inconsistent: the range does not hold the crossing
                atomicOr(&S.ctr->status, 1 << KP_ESTATE);
                resolved(sk, k, sk.lo, lam_t, lam_next);
            }
            S.sel[k] = sk;
        }
        return;
    }
    if (!ovf) {
        bool ok = true;
        const uint32_t key = exact_select(S, P, k, sk.lo, sk.hi, Bfix - sk.above, &ok);
        if (threadIdx.x == 0) {
            if (!ok) atomicOr(&S.ctr->status, 1 << KP_ESTATE);
            resolved(sk, k, key, lam_t, lam_next);
            S.sel[k] = sk;
        }
        return;
    }
    const uint32_t width = sk.hi - sk.lo;
    int sh = bitlen32(width - 1) - 8;
    if (sh < 0) sh = 0;
    const uint32_t lo = sk.lo + ((uint32_t)pick << sh);
    const uint32_t span = sh == 0 ? 1u : (1u << sh);
    const uint32_t hi = (sk.hi - lo) < span ? sk.hi : lo + span;
    if (threadIdx.x == 0) {
        if (round >= MAX_REFINE) {
            atomicOr(&S.ctr->status, 1 << KP_ESTATE);
            resolved(sk, k, lo, lam_t, lam_next);
        } else {
            unresolved(S, sk, lo, hi, s_above, round);
        }
        S.sel[k] = sk;
    }
}

__global__ void select_kernel(Params P, Scratch S, const double *lam, double *lam_next, int round) {
    select_body(P, S, blockIdx.x, lam, lam_next, round);
}

// one block per (instance, knapsack) of a batch
__global__ void batch_select_kernel(BatchDev B, const double *lam, double *lam_next, int round) {
    __shared__ Params sP;
    __shared__ Scratch sS;
    __shared__ int s_skip;
    const int i = B.kinst[blockIdx.x];
    const int64_t ko = B.koff[i];
    if (B.solo[i]) return;  // selected by its own launch
    if (threadIdx.x == 0) {
        sP = B.P[i];
        sS = B.S[i];
        s_skip = round > 0 && sS.ctr->n_unres[round] == 0;
    }
    __syncthreads();
    if (s_skip) return;
    select_body(sP, sS, (int)(blockIdx.x - ko), lam + ko, lam_next + ko, round);
}

constexpr int BWD_USERS = 256;

__global__ void backward_kernel(int64_t N, int M, int W, int K, const double *lam,
                                const uint32_t *x_bits, const double *R, const double *B,
                                const double *upstream, double *grad_lambda, float *grad_p,
                                double *grad_B) {
    const double up = *upstream;
    if (blockIdx.x == 0) {
        for (int k = threadIdx.x; k < K; k += blockDim.x) {
            if (grad_lambda) grad_lambda[k] = up * (B[k] - R[k]);
            if (grad_B) grad_B[k] = up * lam[k];
        }
    }
    if (!grad_p) return;
    // grad_p = up * x*: a chunk of BWD_USERS users (one per thread) is expanded
    // into shared memory, then written out with 16-byte stores by consecutive
    // threads (each chunk starts 16-byte aligned when grad_p does)
    extern __shared__ __align__(16) float stage[];  // [BWD_USERS * M]
    const float upf = (float)up;
    const bool vec = (reinterpret_cast<uintptr_t>(grad_p) & 15u) == 0;
    for (int64_t i0 = (int64_t)blockIdx.x * BWD_USERS; i0 < N; i0 += (int64_t)gridDim.x * BWD_USERS) {
        const int nu = (int)(N - i0 < BWD_USERS ? N - i0 : BWD_USERS);
        const int ne = nu * M;
        if ((int)threadIdx.x < nu) {
            const uint32_t *xw = x_bits + (i0 + threadIdx.x) * W;
            float *row = stage + threadIdx.x * M;
            uint32_t wd = 0u;
            for (int j = 0; j < M; ++j) {
                if ((j & 31) == 0) wd = __ldg(xw + (j >> 5));
                row[j] = ((wd >> (j & 31)) & 1u) ? upf : 0.f;
            }
        }
        __syncthreads();
        float *gp = grad_p + i0 * M;
        if (vec) {
            const int n4 = ne >> 2;
            for (int q = threadIdx.x; q < n4; q += blockDim.x)
                reinterpret_cast<float4 *>(gp)[q] = reinterpret_cast<const float4 *>(stage)[q];
            for (int q = (n4 << 2) + threadIdx.x; q < ne; q += blockDim.x) gp[q] = stage[q];
        } else {
            for (int q = threadIdx.x; q < ne; q += blockDim.x) gp[q] = stage[q];
        }
        __syncthreads();
    }
}

__device__ __forceinline__ bool finite_nonneg(float v) { return v >= 0.f && v <= FLT_MAX; }

__global__ void validate_kernel(Params P, uint32_t *flags) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t bad = 0, maxb = 0;
    const int M = P.M, K = P.K;
    uint32_t maxp = 0;
    for (int64_t q = tid; q < P.N * M; q += stride) {
        const float v = P.p[q];
        if (!finite_nonneg(v)) bad |= 1u;
        else maxp = max(maxp, __float_as_uint(v));
    }
    if (P.layout == KP_B_DENSE) {
        const int64_t tot = P.N * (int64_t)M * K;
        for (int64_t q = tid; q < tot; q += stride) {
            const float v = P.b[q];
            if (!finite_nonneg(v)) bad |= 2u;
            else maxb = max(maxb, __float_as_uint(v));
        }
    } else {
        for (int64_t i = tid; i < P.N; i += stride) {
            const int64_t e0 = P.uoff[i], e1 = P.uoff[i + 1];
            int64_t e = e0;
            for (int j = 0; j < M; ++j) {
                const int c = P.innz[i * M + j];
                int prev = -1;
                for (int q = 0; q < c; ++q, ++e) {
                    if (e >= e1) break;
                    const int k = P.kidx[e];
                    if (k < 0 || k >= K || k <= prev) bad |= 8u;
                    prev = k;
                    const float v = P.val[e];
                    if (!finite_nonneg(v)) bad |= 2u;
                    else maxb = max(maxb, __float_as_uint(v));
                }
            }
            if (e != e1 || e0 < 0) bad |= 4u;
        }
        uint32_t cmin = 0xffffffffu, cmax = 0u;
        for (int64_t q = tid; q < P.N * M; q += stride) {
            const uint32_t c = P.innz[q];
            cmin = min(cmin, c);
            cmax = max(cmax, c);
        }
        atomicMin(&flags[3], cmin);
        atomicMax(&flags[4], cmax);
    }
    for (int64_t k = tid; k < K; k += stride) {
        const double Bk = P.B[k];
        if (!(Bk > 0.0) || !(Bk < 1e300)) bad |= 16u;
    }
    if (bad) atomicOr(&flags[0], bad);
    if (maxb) atomicMax(&flags[1], maxb);
    if (maxp) atomicMax(&flags[2], maxp);
}

int sm_count() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

// For every user with at most 32 entries: bit e of .x set iff entry e has
// b > 0 and another item of the same user has an entry with the same knapsack
// and b > 0; .y lists up to PAIRS_MAX knapsacks that exactly two items of the
// user use as (first entry, second entry).  Knapsacks used by three or more
// items, and pairs beyond PAIRS_MAX, are counted in *count and, if
// rare != nullptr, listed as (user << 5) | first entry (at most cap of them).
__global__ void shmask_kernel(Params P, uint2 *shmask, unsigned long long *rare, int64_t cap,
                              unsigned long long *count) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P.N; i += stride) {
        const int64_t e0 = P.uoff[i];
        const int64_t nnz = P.uoff[i + 1] - e0;
        if (nnz > 32) {
            shmask[i] = make_uint2(0u, 0u);
            continue;
        }
        int owner[32];
        int e = 0;
        for (int j = 0; j < P.M; ++j) {
            const int c = P.innz[i * P.M + j];
            for (int q = 0; q < c && e < 32; ++q) owner[e++] = j;
        }
        uint32_t m = 0, pairs = 0;
        int np = 0;
        for (int a = 0; a < (int)nnz; ++a) {
            if (!(P.val[e0 + a] > 0.f)) continue;
            const int ka = P.kidx[e0 + a];
            int users = 1;  // entries of knapsack ka with b > 0 (one per item)
            int partner = -1;
            bool earlier = false;
            for (int b = 0; b < (int)nnz; ++b)
                if (b != a && P.kidx[e0 + b] == ka && P.val[e0 + b] > 0.f) {
                    if (owner[b] != owner[a]) ++users;
                    if (b < a) earlier = true;
                    partner = b;
                }
            if (users >= 2) {
                m |= 1u << a;
                if (!earlier) {
                    if (users == 2 && np < PAIRS_MAX) {
                        pairs |= ((uint32_t)a | ((uint32_t)partner << 5)) << (10 * np);
                        ++np;
                    } else {
                        const unsigned long long slot = atomicAdd(count, 1ull);
                        if (rare && (int64_t)slot < cap) rare[slot] = ((unsigned long long)i << 5) | (unsigned)a;
                    }
                }
            }
        }
        shmask[i] = make_uint2(m, pairs | ((uint32_t)np << 30));
    }
}

}  // namespace

cudaError_t launch_shmask(const Params &P, uint2 *shmask, unsigned long long *rare, int64_t cap,
                          unsigned long long *count, cudaStream_t st) {
    shmask_kernel<<<sm_count() * 8, 256, 0, st>>>(P, shmask, rare, cap, count);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const Params &P, const Scratch &S, const double *lambda, double *R,
                            double *dual, double *primal, double *g, double alpha,
                            double *lambda_next, cudaStream_t st) {
    finalize_kernel<<<1, 256, 0, st>>>(P, S, lambda, R, dual, primal, g, alpha, lambda_next,
                                       lambda_next != nullptr);
    return cudaGetLastError();
}

cudaError_t launch_batch_finalize(const BatchDev &B, const double *lam, double *R, double *dual,
                                  double *primal, double alpha, double *lam_next, cudaStream_t st) {
    batch_finalize_kernel<<<B.count, 256, 0, st>>>(B, lam, R, dual, primal, alpha, lam_next,
                                                   lam_next != nullptr);
    return cudaGetLastError();
}

cudaError_t launch_batch_select(const BatchDev &B, int64_t totK, const double *lam,
                                double *lam_next, int round, cudaStream_t st) {
    batch_select_kernel<<<(unsigned)totK, 256, 0, st>>>(B, lam, lam_next, round);
    return cudaGetLastError();
}

// Bucketed Reduce of Sec. 5.2.  Prep: every knapsack to state 2 with its
// bucket width Delta_k = delta lambda_k^t (delta where lambda_k^t = 0), the
// bucket masses cleared, the re-run pass of BUCKET_ROUND enabled.
__global__ void bucket_prep_kernel(Params P, Scratch S, const double *lam, double delta) {
    const int K = P.K;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < K * NSUB; q += gridDim.x * blockDim.x) {
        S.subhist[q] = 0ull;
        if (q < K) {
            const double l = lam[q];
            const float dl = (float)(l > 0.0 ? delta * l : delta);
            S.sel[q].state = 2;
            S.sel[q].bdelta = dl > FLT_MIN ? dl : FLT_MIN;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) S.ctr->n_unres[BUCKET_ROUND] = K;
}

// Select: walking down from the highest bucket, the first bucket whose mass
// takes the cumulative mass above B_k holds the threshold; inside it the mass
// is taken as uniform over the bucket's range [lo, hi) and lambda_k^{t+1} is
// the point where the cumulative mass reaches B_k (linear interpolation),
// clamped to the bucket and to lambda >= 0.  No bucket crosses B_k (the whole
// emitted mass is within the budget): lambda_k^{t+1} = 0, as in Algorithm 4.
// Integer fixed-point masses locate the bucket exactly; the interpolation is FP64.
__global__ void bucket_select_kernel(Params P, Scratch S, const double *lam, double *lam_next) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P.K) return;
    const unsigned long long *h = S.subhist + (size_t)k * NSUB;
    const unsigned long long Bfix = budget_fixed(P.B[k], P.fixs);
    unsigned long long A = 0ull;
    int hit = -1;
    for (int b = NSUB - 1; b >= 1; --b) {
        const unsigned long long m = h[b];
        if (A + m > Bfix) {
            hit = b;
            break;
        }
        A += m;
    }
    double out = 0.0;
    if (hit >= 0) {
        const double lt = (double)(float)lam[k], dl = (double)S.sel[k].bdelta;
        const int id = hit - 128;
        double lo, hi;
        if (id == 0) {
            lo = lt - dl;
            hi = lt + dl;
        } else if (id > 0) {
            lo = lt + ldexp(dl, id - 1);
            hi = lt + ldexp(dl, id);
        } else {
            lo = lt - ldexp(dl, -id);
            hi = lt - ldexp(dl, -id - 1);
        }
        const double f = (double)(Bfix - A) / (double)h[hit];
        out = hi - f * (hi - lo);
        out = fmin(fmax(out, lo), hi);
        out = fmax(out, 0.0);
    }
    lam_next[k] = out;
    S.sel[k].state = 0;
    if (k == 0) S.ctr->n_unres[BUCKET_ROUND] = 0;
}

cudaError_t launch_bucket_prep(const Params &P, const Scratch &S, const double *lambda, double delta,
                               cudaStream_t st) {
    const int n = P.K * NSUB;
    bucket_prep_kernel<<<(n + 255) / 256, 256, 0, st>>>(P, S, lambda, delta);
    return cudaGetLastError();
}

cudaError_t launch_bucket_select(const Params &P, const Scratch &S, const double *lambda, double *lambda_next,
                                 cudaStream_t st) {
    bucket_select_kernel<<<(P.K + 127) / 128, 128, 0, st>>>(P, S, lambda, lambda_next);
    return cudaGetLastError();
}

cudaError_t launch_select(const Params &P, const Scratch &S, const double *lambda,
                          double *lambda_next, int round, cudaStream_t st) {
    select_kernel<<<P.K, 256, 0, st>>>(P, S, lambda, lambda_next, round);
    return cudaGetLastError();
}

cudaError_t launch_backward(const Params &P, const double *lambda, const uint32_t *x_bits,
                            const double *R, const double *upstream, double *grad_lambda,
                            float *grad_p, double *grad_B, cudaStream_t st) {
    const int sms = sm_count();
    int64_t blocks = (P.N + BWD_USERS - 1) / BWD_USERS;
    const int64_t cap = (int64_t)sms * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    const size_t smem = (size_t)BWD_USERS * P.M * sizeof(float);  // at most 64 KB (M <= 64)
    static bool attr = false;  // once, before any stream capture
    if (!attr) {
        cudaFuncSetAttribute(backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)((size_t)BWD_USERS * KP_MAX_M * sizeof(float)));
        attr = true;
    }
    backward_kernel<<<(int)blocks, BWD_USERS, smem, st>>>(P.N, P.M, P.W, P.K, lambda, x_bits, R, P.B,
                                                          upstream, grad_lambda, grad_p, grad_B);
    return cudaGetLastError();
}

cudaError_t launch_validate(const Params &P, uint32_t *flags, cudaStream_t st) {
    const int sms = sm_count();
    validate_kernel<<<sms * 4, 256, 0, st>>>(P, flags);
    return cudaGetLastError();
}

}  // namespace kp
