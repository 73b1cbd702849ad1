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
// digit first:
//   1. a pass over all users computes and stores the keys, the consumption R
//      of the given x and the smallest and largest key;
//   2. a one-block kernel finds the knapsacks over budget (the only ones the
//      selection needs) and skips the leading key bits that all users share;
//   3. level by level, a pass over the users whose key matches the digits
//      found so far sums, per value of the next digit, the number of users and
//      the exact fixed-point consumption of every knapsack over budget; a
//      one-block kernel takes the largest digit at which some knapsack still
//      short of its excess reaches it (knapsacks covered by the lower digits
//      drop out, the others keep the rest of their excess).  The users that
//      match are listed, so that each level reads only the previous level's
//      matches;
//   4. a last pass resets the users whose key is at most t's and sums the
//      consumption they release.
// Digits have 3 to 8 bits, as many as the per-digit sums of the knapsacks over
// budget allow in shared memory.
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

constexpr int PP_THREADS = 512;    // user passes
constexpr int PPF_THREADS = 1024;  // one-block kernels
constexpr int PP_MIN_DBITS = 3, PP_MAX_DBITS = 8;
constexpr int PP_BIN_WORDS = 12288;  // 96 KB of per-digit sums (more when 8 (K+1) words need it)

struct PPState {
    unsigned long long prefix_hi, prefix_lo;  // digits of t's composite key found so far
    unsigned long long umin, umax;            // smallest and largest key
    unsigned long long nlist[2];              // lengths of the two match lists
    unsigned long long count;                 // users reset
    int32_t phase;                            // 0 searching, 1 feasible as given, 2 t found
    int32_t cut;                              // composite bits below cut are still open
    int32_t dbits;                            // bits per digit
    int32_t nact;                             // knapsacks over budget
    int32_t pad[2];
};

struct PPWork {
    unsigned long long *ukey;     // [N] order-preserving bits of q_i
    int64_t *list[2];             // [N] each: users matching the digits of a level
    unsigned long long *bins;     // [nd][nact] consumption per digit, then [nd] user counts
    unsigned long long *Rfix;     // [K] consumption of the given x
    unsigned long long *removed;  // [K] consumption of the users reset
    unsigned long long *need;     // [nact] excess not yet covered (0: covered)
    int32_t *kslot;               // [K] slot of a knapsack over budget, -1 otherwise
    PPState *st;
    int32_t *status;              // bit kp_status of errors (the handle's device status)
};

// order-preserving unsigned image of a double; -0 and +0 compare equal and
// map to the same key
__device__ __forceinline__ unsigned long long ordered_key(double q) {
    const unsigned long long u = q == 0.0 ? 0ull : (unsigned long long)__double_as_longlong(q);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

__device__ __forceinline__ u128 composite(unsigned long long key, int64_t i, int ib) {
    return (((u128)key) << ib) | (u128)(uint64_t)i;
}

__device__ __forceinline__ u128 prefix_of(const PPState &s) {
    return (((u128)s.prefix_hi) << 64) | (u128)s.prefix_lo;
}

__device__ __forceinline__ uint64_t user_x(const Params &P, const uint32_t *x, int64_t i) {
    uint64_t xm = x[i * P.W];
    if (P.W > 1) xm |= (uint64_t)x[i * P.W + 1] << 32;
    return P.M == 64 ? xm : xm & ((1ull << P.M) - 1ull);
}

// q_i: items in ascending j, the knapsacks of an item in ascending k
// First entry of item j of user i (CSR): with the same number creg of entries
// per item it is computed, otherwise the counts of the items before j are summed.
__device__ __forceinline__ int64_t item_entry(const Params &P, int64_t i, int j, int64_t &e_walk, int &j_walk) {
    if (P.creg > 0) return P.uoff0 + (i * P.M + j) * (int64_t)P.creg;
    while (j_walk < j) e_walk += P.innz[i * P.M + j_walk++];
    return e_walk;
}

template <int LAYOUT>
__device__ double group_profit(const Params &P, const double *lambda, uint64_t xm, int64_t i) {
    double q = 0.0;
    int64_t ew = LAYOUT == KP_B_CSR && P.creg == 0 ? P.uoff[i] : 0;
    int jw = 0;
    uint64_t r = xm;
    while (r) {  // the selected items, ascending j
        const int j = __ffsll((long long)r) - 1;
        r &= r - 1;
        q = __dadd_rn(q, (double)P.p[i * P.M + j]);
        if (LAYOUT == KP_B_CSR) {
            const int64_t e = item_entry(P, i, j, ew, jw);
            const int n = P.creg > 0 ? P.creg : (int)P.innz[i * P.M + j];
            for (int c = 0; c < n; ++c)
                q = __dsub_rn(q, __dmul_rn(lambda[P.kidx[e + c]], (double)P.val[e + c]));
        } else {
            const float *bj = P.b + (i * P.M + j) * (int64_t)P.K;
            for (int k = 0; k < P.K; ++k) q = __dsub_rn(q, __dmul_rn(lambda[k], (double)bj[k]));
        }
    }
    return q;
}

// adds the user's consumption of knapsack k to counter base + slot[k] of the
// shared sums (every k when slot is NULL; knapsacks with slot -1 are skipped)
template <int LAYOUT>
__device__ void add_consumption(const Params &P, uint64_t xm, int64_t i, const kp::SFix &bin, int base,
                                const int32_t *slot) {
    int64_t ew = LAYOUT == KP_B_CSR && P.creg == 0 ? P.uoff[i] : 0;
    int jw = 0;
    uint64_t r = xm;
    while (r) {
        const int j = __ffsll((long long)r) - 1;
        r &= r - 1;
        if (LAYOUT == KP_B_CSR) {
            const int64_t e = item_entry(P, i, j, ew, jw);
            const int n = P.creg > 0 ? P.creg : (int)P.innz[i * P.M + j];
            for (int c = 0; c < n; ++c) {
                const int k = P.kidx[e + c];
                const int s = slot ? slot[k] : k;
                if (s < 0) continue;
                const uint32_t m = kp::bmass(P.val[e + c], P.bscale);
                if (m) bin.add(base + s, m);
            }
        } else {
            const float *bj = P.b + (i * P.M + j) * (int64_t)P.K;
            for (int k = 0; k < P.K; ++k) {
                const int s = slot ? slot[k] : k;
                if (s < 0) continue;
                const uint32_t m = kp::bmass(bj[k], P.bscale);
                if (m) bin.add(base + s, m);
            }
        }
    }
}

__device__ __forceinline__ unsigned long long warp_min(unsigned long long v) {
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long u = __shfl_xor_sync(0xffffffffu, v, o);
        v = u < v ? u : v;
    }
    return v;
}

__device__ __forceinline__ unsigned long long warp_max(unsigned long long v) {
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long u = __shfl_xor_sync(0xffffffffu, v, o);
        v = u > v ? u : v;
    }
    return v;
}

// Step 1: every user's key, the consumption of the given x, the key range.
// The loop bound is uniform per warp (warp-wide min / max).
template <int LAYOUT>
__global__ void __launch_bounds__(PP_THREADS) pp_keys_kernel(const Params P, const double *lambda,
                                                             const uint32_t *x, PPWork w) {
    extern __shared__ unsigned long long smem_pp[];
    const kp::SFix sR{(uint32_t *)smem_pp, P.K};  // [K] consumption (word pairs)
    for (int k = threadIdx.x; k < P.K; k += blockDim.x) sR.zero(k);
    __syncthreads();
    unsigned long long lo = ~0ull, hi = 0ull;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t b0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); b0 < P.N; b0 += stride) {
        const int64_t i = b0 + lane;
        if (i < P.N) {
            const uint64_t xm = user_x(P, x, i);
            const unsigned long long key = ordered_key(xm ? group_profit<LAYOUT>(P, lambda, xm, i) : 0.0);
            w.ukey[i] = key;
            lo = key < lo ? key : lo;
            hi = key > hi ? key : hi;
            if (xm) add_consumption<LAYOUT>(P, xm, i, sR, 0, nullptr);
        }
    }
    lo = warp_min(lo);
    hi = warp_max(hi);
    if (lane == 0 && hi >= lo) {  // the warp saw a user
        atomicMin(&w.st->umin, lo);
        atomicMax(&w.st->umax, hi);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < P.K; k += blockDim.x) {
        const unsigned long long v = sR.get(k);
        if (v) atomicAdd(&w.Rfix[k], v);
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

// Step 2: knapsacks over budget get consecutive slots; the selection starts
// below the leading composite bits common to the smallest and largest key.
__global__ void __launch_bounds__(PPF_THREADS) pp_start_kernel(PPWork w, const double *B, int K, int fixs,
                                                               int ib, int bin_words) {
    if (threadIdx.x != 0) return;
    PPState &s = *w.st;
    int nact = 0;
    for (int k = 0; k < K; ++k) {
        const unsigned long long R = w.Rfix[k];
        unsigned long long fb;
        if (budget_units(B[k], fixs, &fb) && R > fb) {
            w.need[nact] = R - fb;
            w.kslot[k] = nact++;
        } else {
            w.kslot[k] = -1;
        }
    }
    s.nact = nact;
    if (nact == 0) {
        s.phase = 1;
        return;
    }
    const unsigned long long diff = s.umin ^ s.umax;
    const int common = diff ? __clzll((long long)diff) : 64;  // leading key bits shared by all users
    const int T = 64 + ib;
    s.cut = T - common;
    const unsigned long long top = common >= 64 ? s.umin : common ? (s.umin & ~(~0ull >> common)) : 0ull;
    const u128 pre = composite(top, 0, ib);
    s.prefix_hi = (unsigned long long)(pre >> 64);
    s.prefix_lo = (unsigned long long)pre;
    int d = PP_MAX_DBITS;
    while (d > PP_MIN_DBITS && ((size_t)1 << d) * (size_t)(nact + 1) > (size_t)bin_words) --d;
    s.dbits = d;
    s.phase = 0;
}

// Step 3, one level: users whose composite key matches the digits found so far
// are counted, and their consumption of every knapsack over budget summed,
// per value of the next digit.  Levels 0 and 1 scan all users, level l >= 2
// the users listed by level l - 1; levels >= 1 list their matches.
template <int LAYOUT>
__global__ void __launch_bounds__(PP_THREADS) pp_level_kernel(const Params P, const uint32_t *x, PPWork w,
                                                              int level, int ib) {
    extern __shared__ unsigned long long smem_pp[];  // [nd][nact] sums, [nd] counts (word pairs), then slots
    const PPState s = *w.st;
    if (s.phase != 0) return;
    const int nact = s.nact, nd = 1 << s.dbits, nb = nd * nact + nd;
    const kp::SFix sbin{(uint32_t *)smem_pp, nb};
    int32_t *slot = (int32_t *)(smem_pp + nb);
    for (int q = threadIdx.x; q < nb; q += blockDim.x) sbin.zero(q);
    for (int k = threadIdx.x; k < P.K; k += blockDim.x) slot[k] = w.kslot[k];
    __syncthreads();
    const int cut = s.cut, pos = cut > s.dbits ? cut - s.dbits : 0;
    const unsigned dmask = (1u << (cut - pos)) - 1u;
    const u128 pre = prefix_of(s) >> cut;
    const bool all = level <= 1;
    // (selects instead of indexing keep the structures in registers)
    const bool odd = level & 1;
    const int64_t n = all ? P.N : (int64_t)(odd ? s.nlist[0] : s.nlist[1]);
    const int64_t *in = odd ? w.list[0] : w.list[1];
    int64_t *out = odd ? w.list[1] : w.list[0];
    unsigned long long *nout = odd ? &w.st->nlist[1] : &w.st->nlist[0];
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t b0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); b0 < n; b0 += stride) {
        const int64_t r = b0 + lane;
        int64_t i = 0;
        bool match = false;
        u128 c = 0;
        if (r < n) {
            i = all ? r : in[r];
            c = composite(w.ukey[i], i, ib);
            match = (c >> cut) == pre;
        }
        if (level >= 1) {  // append the matches to this level's list
            const unsigned ball = __ballot_sync(0xffffffffu, match);
            unsigned long long base = 0;
            if (lane == 0 && ball) base = atomicAdd(nout, (unsigned long long)__popc(ball));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (match) out[base + __popc(ball & ((1u << lane) - 1u))] = i;
        }
        if (!match) continue;
        const int d = (int)((unsigned)(uint64_t)(c >> pos) & dmask);
        sbin.add(nd * nact + d, 1u);
        const uint64_t xm = user_x(P, x, i);
        if (xm) add_consumption<LAYOUT>(P, xm, i, sbin, d * nact, slot);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < nb; q += blockDim.x) {
        const unsigned long long v = sbin.get(q);
        if (v) atomicAdd(&w.bins[q], v);
    }
}

// Step 3, the digit of a level: the largest digit at which a knapsack whose
// excess is not yet covered reaches it; updates the excesses, the digits of t
// and the bins (zeroed for the next level).
__global__ void __launch_bounds__(PPF_THREADS) pp_select_kernel(PPWork w, int level) {
    __shared__ int s_dstar;
    __shared__ unsigned long long s_at;
    __shared__ PPState s;
    if (threadIdx.x == 0) {
        s = *w.st;
        s_dstar = -1;
    }
    __syncthreads();
    if (s.phase != 0) return;
    const int nact = s.nact, nd = 1 << s.dbits;
    const unsigned long long *cnt = w.bins + (size_t)nd * nact;
    for (int a = threadIdx.x; a < nact; a += blockDim.x) {
        const unsigned long long need = w.need[a];
        if (!need) continue;
        unsigned long long cum = 0;
        int da = -1;
        for (int d = 0; d < nd && da < 0; ++d) {
            cum += w.bins[(size_t)d * nact + a];
            if (cum >= need) da = d;
        }
        if (da < 0) {  // the excess is always reached inside the matching range
            atomicOr(w.status, 1 << KP_ESTATE);
            da = nd - 1;
        }
        atomicMax(&s_dstar, da);
    }
    __syncthreads();
    const int ds = s_dstar;
    if (ds < 0) {  // some knapsack always keeps an uncovered excess
        if (threadIdx.x == 0) {
            atomicOr(w.status, 1 << KP_ESTATE);
            w.st->phase = 3;
        }
        return;
    }
    for (int a = threadIdx.x; a < nact; a += blockDim.x) {
        unsigned long long below = 0;
        for (int d = 0; d < ds; ++d) below += w.bins[(size_t)d * nact + a];
        const unsigned long long need = w.need[a];
        if (need) w.need[a] = below >= need ? 0ull : need - below;
    }
    if (threadIdx.x == 0) s_at = cnt[ds];
    __syncthreads();
    for (int q = threadIdx.x; q < nd * nact + nd; q += blockDim.x) w.bins[q] = 0ull;
    if (threadIdx.x == 0) {
        const int pos = s.cut > s.dbits ? s.cut - s.dbits : 0;
        if (pos == 0 && s_at != 1ull) atomicOr(w.status, 1 << KP_ESTATE);  // t is one user
        const u128 pre = prefix_of(s) | (((u128)ds) << pos);
        w.st->prefix_hi = (unsigned long long)(pre >> 64);
        w.st->prefix_lo = (unsigned long long)pre;
        w.st->cut = pos;
        if (level & 1) w.st->nlist[0] = 0ull;  // the next level's list
        else w.st->nlist[1] = 0ull;
        if (pos == 0) w.st->phase = 2;
    }
}

// Step 4: resets every user at or before t, counts them and sums the
// consumption they release
template <int LAYOUT>
__global__ void __launch_bounds__(PP_THREADS) pp_clear_kernel(const Params P, uint32_t *x, PPWork w, int ib) {
    extern __shared__ unsigned long long smem_pp[];
    const kp::SFix sR{(uint32_t *)smem_pp, P.K};  // [K] released consumption (word pairs)
    if (w.st->phase != 2) return;
    for (int k = threadIdx.x; k < P.K; k += blockDim.x) sR.zero(k);
    __syncthreads();
    const u128 t = prefix_of(*w.st);
    unsigned long long n = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P.N; i += stride) {
        if (composite(w.ukey[i], i, ib) > t) continue;
        ++n;
        const uint64_t xm = user_x(P, x, i);
        if (!xm) continue;
        add_consumption<LAYOUT>(P, xm, i, sR, 0, nullptr);
        for (int q = 0; q < P.W; ++q) x[i * P.W + q] = 0u;
    }
    for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    if ((threadIdx.x & 31) == 0 && n) atomicAdd(&w.st->count, n);
    __syncthreads();
    for (int k = threadIdx.x; k < P.K; k += blockDim.x) {
        const unsigned long long v = sR.get(k);
        if (v) atomicAdd(&w.removed[k], v);
    }
}

// the number of users reset and the consumption of the returned x, which must
// fit every budget
__global__ void __launch_bounds__(PPF_THREADS) pp_output_kernel(PPWork w, const double *B, int K, int fixs,
                                                                int64_t *reset, double *R_after) {
    const int phase = w.st->phase;
    if (threadIdx.x == 0) {
        if (phase != 1 && phase != 2) atomicOr(w.status, 1 << KP_ESTATE);
        if (reset) *reset = phase == 2 ? (int64_t)w.st->count : 0;
    }
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        const unsigned long long r = w.Rfix[k] - w.removed[k];
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

template <class F>
int grid_for(F f, size_t smem, int sms, int64_t work) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, f, PP_THREADS, smem) != cudaSuccess || occ < 1)
        return 0;
    const int64_t need = (work + PP_THREADS - 1) / PP_THREADS;
    const int64_t full = (int64_t)sms * occ;
    return (int)(need < full ? (need > 0 ? need : 1) : full);
}

}  // namespace

extern "C" {

kp_status kp_postprocess(kp_problem *h, const double *lambda, uint32_t *x_bits, int64_t *reset,
                         double *R_after, void *stream) {
    if (!h || h->P.N < 1 || !lambda || !x_bits) {
        kp::set_last_error("kp_postprocess: NULL argument");
        return KP_EINVAL;
    }
    const Params &P = h->P;
    cudaStream_t st = (cudaStream_t)stream;
    const int K = P.K, ib = index_bits(P.N), T = 64 + ib;
    const int bin_words = PP_BIN_WORDS > 8 * (K + 1) ? PP_BIN_WORDS : 8 * (K + 1);
    // every level fixes at least PP_MIN_DBITS composite bits
    const int levels = (T + PP_MIN_DBITS - 1) / PP_MIN_DBITS;
    const size_t words = (size_t)P.N * 3 + (size_t)bin_words + 3 * (size_t)K + ((size_t)K + 1) / 2 +
                         sizeof(PPState) / 8;
    // the keys and lists (24 N bytes) stay with the handle after the first call
    cudaError_t e = cudaSuccess;
    if (h->ppwords < words) {
        if (h->ppbuf) {
            e = cudaStreamSynchronize(st);  // the previous scratch may still be in use
            if (e == cudaSuccess) e = cudaFree(h->ppbuf);
            h->ppbuf = nullptr;
            h->ppwords = 0;
        }
        void *p = nullptr;
        if (e == cudaSuccess) e = cudaMalloc(&p, words * sizeof(unsigned long long));
        if (e != cudaSuccess) {
            kp::set_last_error(cudaGetErrorString(e));
            return e == cudaErrorMemoryAllocation ? KP_ENOMEM : KP_ECUDA;
        }
        h->ppbuf = static_cast<unsigned long long *>(p);
        h->ppwords = words;
    }
    unsigned long long *buf = h->ppbuf;
    PPWork w;
    w.ukey = buf;
    w.list[0] = (int64_t *)(buf + P.N);
    w.list[1] = (int64_t *)(buf + 2 * (size_t)P.N);
    w.bins = buf + 3 * (size_t)P.N;
    w.Rfix = w.bins + bin_words;
    w.removed = w.Rfix + K;
    w.need = w.removed + K;
    w.st = (PPState *)(w.need + K);
    w.kslot = (int32_t *)(w.st + 1);
    w.status = &h->S.ctr->status;
    const size_t zero_from = 3 * (size_t)P.N;
    e = cudaMemsetAsync(w.bins, 0, (words - zero_from) * sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(&w.st->umin, 0xff, sizeof(unsigned long long), st);
    const bool csr = P.layout == KP_B_CSR;
    auto keys = csr ? pp_keys_kernel<KP_B_CSR> : pp_keys_kernel<KP_B_DENSE>;
    auto lvl = csr ? pp_level_kernel<KP_B_CSR> : pp_level_kernel<KP_B_DENSE>;
    auto clr = csr ? pp_clear_kernel<KP_B_CSR> : pp_clear_kernel<KP_B_DENSE>;
    const size_t smem_k = (size_t)K * sizeof(unsigned long long);
    const size_t smem_l = (size_t)bin_words * sizeof(unsigned long long) + (size_t)K * sizeof(int32_t);
    int sms = 0;
    if (e == cudaSuccess) e = cudaFuncSetAttribute(keys, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_k);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(lvl, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_l);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(clr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_k);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    int gk = 0, gl = 0, gc = 0;
    if (e == cudaSuccess) {
        gk = grid_for(keys, smem_k, sms, P.N);
        gl = grid_for(lvl, smem_l, sms, P.N);
        gc = grid_for(clr, smem_k, sms, P.N);
        if (!gk || !gl || !gc) e = cudaErrorInvalidConfiguration;
    }
    if (e == cudaSuccess) {
        keys<<<gk, PP_THREADS, smem_k, st>>>(P, lambda, x_bits, w);
        pp_start_kernel<<<1, 32, 0, st>>>(w, P.B, K, P.fixs, ib, bin_words);
        e = cudaGetLastError();
        for (int L = 0; L < levels && e == cudaSuccess; ++L) {
            lvl<<<gl, PP_THREADS, smem_l, st>>>(P, x_bits, w, L, ib);
            pp_select_kernel<<<1, PPF_THREADS, 0, st>>>(w, L);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) {
            clr<<<gc, PP_THREADS, smem_k, st>>>(P, x_bits, w, ib);
            pp_output_kernel<<<1, PPF_THREADS, 0, st>>>(w, P.B, K, P.fixs, reset, R_after);
            e = cudaGetLastError();
        }
    }
    if (e != cudaSuccess) {
        kp::set_last_error(cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? KP_ENOMEM : KP_ECUDA;
    }
    return KP_OK;
}

}  // extern "C"
