// kp_postprocess.cu -- post-processing for feasibility (Sec. 5.4) on the device.
//
// Decisions x taken at dual multipliers lambda may overfill some knapsacks.
// Sec. 5.4 then resets users, taken in non-decreasing order of their
// cost-adjusted group profit
//     q_i = sum_{j : x_ij = 1} (p_ij - sum_k lambda_k b_ijk)
// (equal q_i: lower user index first), until no knapsack exceeds its budget.
// With b >= 0 the consumption only falls as users are reset, so the result is
// the shortest prefix of that order whose consumption covers the excess
// D_k = R_k - B_k of every knapsack, and the users reset are exactly those at
// or before the prefix's last user t.
//
// The N users are not sorted.  t is found by a radix selection over the
// composite key (order-preserving bits of q_i, user index), most significant
// digit first.  At each level one pass over the users whose key matches the
// digits found so far accumulates, for every value d of the next digit, the
// number of users and the exact fixed-point consumption of every knapsack;
// a one-block kernel then takes the largest digit at which the cumulative
// consumption of some knapsack still short of its excess reaches that excess.
// Knapsacks covered by the lower digits drop out, the others keep the rest of
// their excess.  After the last level a pass clears the users whose key is at
// most t's.  Each level's digit has 3 or 4 bits (so that the per-digit
// masses of every knapsack fit in shared memory); a 1e8-user instance takes
// 23 levels.
//
// q_i is accumulated in FP64 in item order, then knapsack order, every
// product and sum rounded to nearest: equal inputs give equal keys, and the
// order is that of the exact left-to-right evaluation of the sum above.
// Consumption is summed in the fixed point of the consumption pass (units of
// 2^-fixs, the per-entry rounding of kp_reduce_consumption), so R_after is
// that pass's R of the returned x.
#include <cmath>

#include "kp_device.cuh"
#include "kp_internal.h"

namespace {

using kp::Params;
typedef unsigned __int128 u128;

constexpr int PP_THREADS = 256;   // user passes
constexpr int PPF_THREADS = 1024; // per-level selection (one block)

struct PPState {
    unsigned long long prefix_hi, prefix_lo;  // digits of t's composite key found so far
    unsigned long long count;                 // users placed before the digits found so far
    int32_t phase;                            // 0 searching, 1 feasible as given, 2 t found
    int32_t pad;
};

struct PPWork {
    unsigned long long *ukey;     // [N] order-preserving bits of q_i
    unsigned long long *bins;     // [nd][K] consumption per digit, then [nd] user counts
    unsigned long long *Rfix;     // [K] consumption of the given x
    unsigned long long *removed;  // [K] consumption of the users reset so far
    unsigned long long *need;     // [K] excess not yet covered (0: covered)
    PPState *st;
    int32_t *status;              // bit kp_status of errors (the handle's device status)
};

// order-preserving unsigned image of a double; -0 and +0 compare equal and
// map to the same key
__device__ __forceinline__ unsigned long long ordered_key(double q) {
    const unsigned long long u = q == 0.0 ? 0ull : (unsigned long long)__double_as_longlong(q);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

__device__ __forceinline__ uint64_t user_x(const Params &P, const uint32_t *x, int64_t i) {
    uint64_t xm = x[i * P.W];
    if (P.W > 1) xm |= (uint64_t)x[i * P.W + 1] << 32;
    return P.M == 64 ? xm : xm & ((1ull << P.M) - 1ull);
}

// q_i: items in ascending j, the knapsacks of an item in ascending k
template <int LAYOUT>
__device__ double group_profit(const Params &P, const double *lambda, uint64_t xm, int64_t i) {
    double q = 0.0;
    int64_t e = LAYOUT == KP_B_CSR ? P.uoff[i] : 0;
    for (int j = 0; j < P.M; ++j) {
        const int n = LAYOUT == KP_B_CSR ? (int)P.innz[i * P.M + j] : 0;
        if ((xm >> j) & 1ull) {
            q = __dadd_rn(q, (double)P.p[i * P.M + j]);
            if (LAYOUT == KP_B_CSR) {
                for (int c = 0; c < n; ++c)
                    q = __dsub_rn(q, __dmul_rn(lambda[P.kidx[e + c]], (double)P.val[e + c]));
            } else {
                const float *bj = P.b + (i * P.M + j) * (int64_t)P.K;
                for (int k = 0; k < P.K; ++k) q = __dsub_rn(q, __dmul_rn(lambda[k], (double)bj[k]));
            }
        }
        e += n;
    }
    return q;
}

// adds the user's consumption of every knapsack to bin[k]
template <int LAYOUT>
__device__ void add_consumption(const Params &P, uint64_t xm, int64_t i, unsigned long long *bin) {
    int64_t e = LAYOUT == KP_B_CSR ? P.uoff[i] : 0;
    for (int j = 0; j < P.M; ++j) {
        const int n = LAYOUT == KP_B_CSR ? (int)P.innz[i * P.M + j] : 0;
        if ((xm >> j) & 1ull) {
            if (LAYOUT == KP_B_CSR) {
                for (int c = 0; c < n; ++c) {
                    const unsigned long long m = kp::bmass(P.val[e + c], P.bscale);
                    if (m) atomicAdd(&bin[P.kidx[e + c]], m);
                }
            } else {
                const float *bj = P.b + (i * P.M + j) * (int64_t)P.K;
                for (int k = 0; k < P.K; ++k) {
                    const unsigned long long m = kp::bmass(bj[k], P.bscale);
                    if (m) atomicAdd(&bin[k], m);
                }
            }
        }
        e += n;
    }
}

// One level of the selection: users whose composite key matches the digits
// found so far are counted, and their consumption summed, per value of the
// next digit.  The first level also computes and stores every user's key.
template <int LAYOUT, bool FIRST>
__global__ void __launch_bounds__(PP_THREADS) pp_pass_kernel(const Params P, const double *lambda,
                                                             const uint32_t *x, PPWork w, int level,
                                                             int dbits, int ib) {
    extern __shared__ unsigned long long sbin[];  // [nd][K] masses, then [nd] counts
    if (!FIRST && w.st->phase != 0) return;
    const int K = P.K, nd = 1 << dbits, nb = nd * K + nd;
    for (int q = threadIdx.x; q < nb; q += blockDim.x) sbin[q] = 0ull;
    __syncthreads();
    const int T = 64 + ib;
    const int cut = T - dbits * level;  // composite bits below cut are not fixed yet
    const int pos = cut > dbits ? cut - dbits : 0;
    const unsigned dmask = (1u << (cut - pos)) - 1u;
    const u128 pre = FIRST ? (u128)0 : ((((u128)w.st->prefix_hi) << 64) | (u128)w.st->prefix_lo) >> cut;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P.N; i += stride) {
        uint64_t xm = 0;
        unsigned long long key;
        if (FIRST) {
            xm = user_x(P, x, i);
            key = ordered_key(group_profit<LAYOUT>(P, lambda, xm, i));
            w.ukey[i] = key;
        } else {
            key = w.ukey[i];
        }
        const u128 c = (((u128)key) << ib) | (u128)i;
        if (!FIRST) {
            if ((c >> cut) != pre) continue;
            xm = user_x(P, x, i);
        }
        const int d = (int)((unsigned)(uint64_t)(c >> pos) & dmask);
        atomicAdd(&sbin[nd * K + d], 1ull);
        if (xm) add_consumption<LAYOUT>(P, xm, i, sbin + (size_t)d * K);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < nb; q += blockDim.x) {
        const unsigned long long v = sbin[q];
        if (v) atomicAdd(&w.bins[q], v);
    }
}

// Budget B_k in consumption units, rounded down: a consumption r (an integer
// number of units) fits iff r <= floor(B_k 2^fixs).  Returns false when the
// budget exceeds every 64-bit consumption.
__device__ __forceinline__ bool budget_units(double Bk, int fixs, unsigned long long *out) {
    const double Bs = floor(ldexp(Bk, fixs));
    if (!(Bs < 18446744073709551616.0)) return false;
    *out = (unsigned long long)Bs;
    return true;
}

// The digit of this level: the largest digit at which a knapsack whose excess
// is not yet covered reaches it; updates the excesses, the consumption and
// count of the users placed before t, the digits of t and the bins (zeroed
// for the next level).
__global__ void __launch_bounds__(PPF_THREADS) pp_select_kernel(PPWork w, const double *B, int K, int fixs,
                                                                int level, int last, int dbits, int ib) {
    __shared__ int s_phase, s_dstar;
    if (threadIdx.x == 0) {
        s_phase = w.st->phase;
        s_dstar = -1;
    }
    __syncthreads();
    if (s_phase != 0) return;
    const int nd = 1 << dbits;
    unsigned long long *cnt = w.bins + (size_t)nd * K;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        if (level == 0) {
            unsigned long long R = 0;
            for (int d = 0; d < nd; ++d) R += w.bins[(size_t)d * K + k];
            w.Rfix[k] = R;
            unsigned long long fb;
            w.need[k] = budget_units(B[k], fixs, &fb) && R > fb ? R - fb : 0ull;
        }
        const unsigned long long need = w.need[k];
        if (!need) continue;
        unsigned long long cum = 0;
        int dk = -1;
        for (int d = 0; d < nd && dk < 0; ++d) {
            cum += w.bins[(size_t)d * K + k];
            if (cum >= need) dk = d;
        }
        if (dk < 0) {  // the excess is always reached inside the matching range
            atomicOr(w.status, 1 << KP_ESTATE);
            dk = nd - 1;
        }
        atomicMax(&s_dstar, dk);
    }
    __syncthreads();
    const int ds = s_dstar;
    if (ds < 0) {  // no knapsack exceeds its budget (possible at the first level only)
        if (threadIdx.x == 0) {
            if (level > 0) atomicOr(w.status, 1 << KP_ESTATE);
            w.st->phase = 1;
        }
        return;
    }
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        unsigned long long below = 0;
        for (int d = 0; d < ds; ++d) below += w.bins[(size_t)d * K + k];
        const unsigned long long at = w.bins[(size_t)ds * K + k];
        w.removed[k] += below + (last ? at : 0ull);
        const unsigned long long need = w.need[k];
        if (need) w.need[k] = below >= need ? 0ull : need - below;
        for (int d = 0; d < nd; ++d) w.bins[(size_t)d * K + k] = 0ull;
    }
    if (threadIdx.x == 0) {
        unsigned long long c = 0;
        for (int d = 0; d < ds; ++d) c += cnt[d];
        if (last) {
            if (cnt[ds] != 1ull) atomicOr(w.status, 1 << KP_ESTATE);  // t is one user
            c += cnt[ds];
        }
        w.st->count += c;
        const int T = 64 + ib, cut = T - dbits * level, pos = cut > dbits ? cut - dbits : 0;
        const u128 pre = ((((u128)w.st->prefix_hi) << 64) | (u128)w.st->prefix_lo) | (((u128)ds) << pos);
        w.st->prefix_hi = (unsigned long long)(pre >> 64);
        w.st->prefix_lo = (unsigned long long)pre;
        if (last) w.st->phase = 2;
        for (int d = 0; d < nd; ++d) cnt[d] = 0ull;
    }
}

// clears the decisions of every user at or before t
__global__ void __launch_bounds__(PP_THREADS) pp_clear_kernel(PPWork w, int64_t N, int W, int ib, uint32_t *x) {
    if (w.st->phase != 2) return;
    const u128 t = (((u128)w.st->prefix_hi) << 64) | (u128)w.st->prefix_lo;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        const u128 c = (((u128)w.ukey[i]) << ib) | (u128)i;
        if (c <= t)
            for (int q = 0; q < W; ++q) x[i * W + q] = 0u;
    }
}

// the number of users reset and the consumption of the returned x, which must
// fit every budget
__global__ void __launch_bounds__(PPF_THREADS) pp_output_kernel(PPWork w, const double *B, int K, int fixs,
                                                                int64_t *reset, double *R_after) {
    const int phase = w.st->phase;
    if (threadIdx.x == 0) {
        if (phase == 0) atomicOr(w.status, 1 << KP_ESTATE);
        if (reset) *reset = phase == 2 ? (int64_t)w.st->count : 0;
    }
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        const unsigned long long r = w.Rfix[k] - (phase == 2 ? w.removed[k] : 0ull);
        unsigned long long fb;
        if (budget_units(B[k], fixs, &fb) && r > fb) atomicOr(w.status, 1 << KP_ESTATE);
        if (R_after) R_after[k] = ldexp((double)r, -fixs);
    }
}

int index_bits(int64_t N) {
    int ib = 1;
    while (ib < 63 && ((int64_t)1 << ib) < N) ++ib;
    return ib;
}

}  // namespace

namespace kp {

int postprocess_levels(int64_t N, int K, int *dbits_out) {
    const int dbits = (size_t)(16 * K + 16) * sizeof(unsigned long long) <= 96 * 1024 ? 4 : 3;
    if (dbits_out) *dbits_out = dbits;
    const int T = 64 + index_bits(N);
    return (T + dbits - 1) / dbits;
}

}  // namespace kp

extern "C" {

kp_status kp_postprocess(kp_problem *h, const double *lambda, uint32_t *x_bits, int64_t *reset,
                         double *R_after, void *stream) {
    if (!h || h->P.N < 1 || !lambda || !x_bits) {
        kp::set_last_error("kp_postprocess: NULL argument");
        return KP_EINVAL;
    }
    const Params &P = h->P;
    cudaStream_t st = (cudaStream_t)stream;
    const int K = P.K, ib = index_bits(P.N);
    int dbits = 0;
    const int levels = kp::postprocess_levels(P.N, K, &dbits);
    const int nd = 1 << dbits;
    const size_t nb = (size_t)nd * K + nd;
    const size_t smem = nb * sizeof(unsigned long long);
    const size_t words = (size_t)P.N + nb + 3 * (size_t)K + sizeof(PPState) / 8;
    unsigned long long *buf = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&buf, words * sizeof(unsigned long long), st);
    if (e != cudaSuccess) {
        kp::set_last_error(cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? KP_ENOMEM : KP_ECUDA;
    }
    PPWork w;
    w.ukey = buf;
    w.bins = buf + P.N;
    w.Rfix = w.bins + nb;
    w.removed = w.Rfix + K;
    w.need = w.removed + K;
    w.st = (PPState *)(w.need + K);
    w.status = &h->S.ctr->status;
    e = cudaMemsetAsync(w.bins, 0, (words - (size_t)P.N) * sizeof(unsigned long long), st);
    auto pass0 = P.layout == KP_B_CSR ? pp_pass_kernel<KP_B_CSR, true> : pp_pass_kernel<KP_B_DENSE, true>;
    auto passL = P.layout == KP_B_CSR ? pp_pass_kernel<KP_B_CSR, false> : pp_pass_kernel<KP_B_DENSE, false>;
    int sms = 0, occ = 0;
    if (e == cudaSuccess) e = cudaFuncSetAttribute(pass0, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(passL, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, passL, PP_THREADS, smem);
    if (e == cudaSuccess && occ < 1) e = cudaErrorInvalidConfiguration;
    if (e == cudaSuccess) {
        const int64_t need_blocks = (P.N + PP_THREADS - 1) / PP_THREADS;
        const int64_t full = (int64_t)sms * occ;
        const int grid = (int)(need_blocks < full ? need_blocks : full);
        for (int L = 0; L < levels && e == cudaSuccess; ++L) {
            if (L == 0)
                pass0<<<grid, PP_THREADS, smem, st>>>(P, lambda, x_bits, w, 0, dbits, ib);
            else
                passL<<<grid, PP_THREADS, smem, st>>>(P, lambda, x_bits, w, L, dbits, ib);
            pp_select_kernel<<<1, PPF_THREADS, 0, st>>>(w, P.B, K, P.fixs, L, L == levels - 1, dbits, ib);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) {
            pp_clear_kernel<<<grid, PP_THREADS, 0, st>>>(w, P.N, P.W, ib, x_bits);
            pp_output_kernel<<<1, PPF_THREADS, 0, st>>>(w, P.B, K, P.fixs, reset, R_after);
            e = cudaGetLastError();
        }
    }
    const cudaError_t ef = cudaFreeAsync(buf, st);
    if (e == cudaSuccess) e = ef;
    if (e != cudaSuccess) {
        kp::set_last_error(cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? KP_ENOMEM : KP_ECUDA;
    }
    return KP_OK;
}

}  // extern "C"
