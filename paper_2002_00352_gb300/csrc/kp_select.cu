// kp_select.cu -- the small kernels around the user pass:
//   finalize_kernel  ordered FP64 sums of the per-block partials, R_k from
//                    the fixed-point accumulators, the dual objective
//                    (Eq. (5)) and the dual-descent update (Eq. (14)).
//   select_kernel    the Reduce of Algorithm 4 for every knapsack: find the
//                    breakpoint at which the mass accumulated from the top
//                    first exceeds B_k, from the bucket histogram and then
//                    exactly among the buffered breakpoints (radix selection
//                    on the FP32 bit patterns, 8 bits per round).
//   backward_kernel  Danskin gradient of the dual function.
//   validate_kernel  checks of Sec. 2's data assumptions at creation.
#include <cfloat>
#include <cstdint>

#include "kp_device.cuh"
#include "kp_internal.h"

namespace kp {

namespace {

__device__ __forceinline__ int bitlen32(uint32_t x) { return x ? 32 - __clz(x) : 0; }

__device__ __forceinline__ unsigned long long budget_fixed(double Bk, int fixs) {
    double v = ldexp(Bk, fixs);
    if (!(v > 0.0)) return 0ull;
    if (v >= 1.8e19) return ~0ull;
    return (unsigned long long)floor(v);
}

__global__ void finalize_kernel(Params P, Scratch S, const double *lam, double *R, double *dual,
                                double *primal, double *g, double alpha, double *lam_next,
                                int do_dd) {
    const int K = P.K;
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int q = 0; q < S.G; ++q) {
            a += S.dual_part[q];
            b += S.primal_part[q];
        }
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
        const double Rk = (double)S.Rfix[k] * inv;
        S.Rfix[k] = 0ull;
        if (R) R[k] = Rk;
        if (do_dd) {
            const double v = lam[k] + alpha * (Rk - P.B[k]);
            lam_next[k] = v > 0.0 ? v : 0.0;
        }
    }
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
    const float scale = __uint_as_float((uint32_t)(127 + P.fixs) << 23);
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
        for (int gblk = 0; gblk < S.G; ++gblk) {
            const uint32_t cnt = S.bufcnt[(size_t)k * S.G + gblk];
            const uint2 *base = S.buf + ((size_t)k * S.G + gblk) * S.cap_kb;
            for (uint32_t s = threadIdx.x; s < cnt; s += blockDim.x) {
                const uint2 e = base[s];
                const uint32_t off = e.x - clo;
                if (e.x >= clo && off < width) atomicAdd(&h[off >> sh], fixmass(__uint_as_float(e.y), scale));
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

__device__ __forceinline__ void resolved(Scratch &S, SelK &sk, int k, uint32_t key,
                                         double *lam_next) {
    lam_next[k] = key ? (double)__uint_as_float(key) : 0.0;
    if (key) {
        int off = bucket_of(key, sk.ckey) - NB_CENTRE;
        if (off < 0) off = -off;
        int w = off + 1;
        sk.w = w < WMIN ? WMIN : (w > 31 ? 31 : w);
        sk.last_nz_key = key;
    }
    sk.state = 0;
}

__global__ void select_kernel(Params P, Scratch S, const double *lam, double *lam_next, int round) {
    const int k = blockIdx.x;
    __shared__ SelK sk;
    __shared__ unsigned long long row[NSUB];
    __shared__ int s_pick;
    __shared__ unsigned long long s_above;
    if (threadIdx.x == 0) sk = S.sel[k];
    __syncthreads();
    if (round > 0 && sk.state != 1) return;
    const unsigned long long Bfix = budget_fixed(P.B[k], P.fixs);
    const int nrow = round == 0 ? NB : NSUB;
    unsigned long long *grow = round == 0 ? S.hist + (size_t)k * NB : S.subhist + (size_t)k * NSUB;
    for (int q = threadIdx.x; q < nrow; q += blockDim.x) {
        row[q] = grow[q];
        grow[q] = 0ull;
    }
    __syncthreads();
    const uint32_t ovf = S.ovf[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        S.ovf[k] = 0u;
        if (ovf) atomicAdd(&S.ctr->stats[2], 1ull);
        // scan from the top for the bucket where the accumulated mass first exceeds B_k
        unsigned long long above = round == 0 ? 0ull : sk.above;
        const unsigned long long need_total = Bfix;
        int pick = -1;
        unsigned long long acc = above;
        for (int b = nrow - 1; b >= 0; --b) {
            if (acc + row[b] > need_total || (acc + row[b] < acc)) {
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
        // the whole mass fits: lambda_k = 0 (round 0), or an inconsistent refine
        if (threadIdx.x == 0) {
            if (round == 0) {
                lam_next[k] = 0.0;
                sk.state = 0;
                atomicAdd(&S.ctr->stats[1], 1ull);
            } else {
                atomicOr(&S.ctr->status, 1 << KP_ESTATE);
                lam_next[k] = sk.lo ? (double)__uint_as_float(sk.lo) : 0.0;
                sk.state = 0;
            }
            S.sel[k] = sk;
        }
        return;
    }
    // key range of the picked bucket
    uint32_t lo, hi;
    if (round == 0) {
        const long long c = (long long)sk.ckey;
        long long l, h;
        if (pick == NB_CENTRE) {
            l = c;
            h = c + 1;
        } else if (pick > NB_CENTRE) {
            const int e = pick - NB_CENTRE - 1;
            l = c + (1ll << e);
            h = c + (2ll << e);
        } else {
            const int e = NB_CENTRE - 1 - pick;
            l = c - (2ll << e) + 1;
            h = c - (1ll << e) + 1;
        }
        if (l < 0) l = 0;
        if (h > 0x7F800000ll) h = 0x7F800000ll;
        if (h <= l) h = l + 1;
        lo = (uint32_t)l;
        hi = (uint32_t)h;
    } else {
        const uint32_t width = sk.hi - sk.lo;
        int sh = bitlen32(width - 1) - 8;
        if (sh < 0) sh = 0;
        lo = sk.lo + ((uint32_t)pick << sh);
        const uint32_t span = sh == 0 ? 1u : (1u << sh);
        hi = (sk.hi - lo) < span ? sk.hi : lo + span;
    }
    const unsigned long long above = s_above;
    int off = pick - NB_CENTRE;
    if (off < 0) off = -off;
    const bool in_window = round == 0 ? (off <= sk.w) : true;
    if (in_window && !ovf) {
        bool ok = true;
        const uint32_t key = exact_select(S, P, k, lo, hi, Bfix - above, &ok);
        if (threadIdx.x == 0) {
            if (!ok) atomicOr(&S.ctr->status, 1 << KP_ESTATE);
            resolved(S, sk, k, key, lam_next);
            S.sel[k] = sk;
        }
        return;
    }
    if (threadIdx.x == 0) {
        if (round >= MAX_REFINE) {
            atomicOr(&S.ctr->status, 1 << KP_ESTATE);
            resolved(S, sk, k, lo, lam_next);
        } else {
            sk.state = 1;
            sk.lo = lo;
            sk.hi = hi;
            sk.above = above;
            atomicAdd(&S.ctr->n_unres[round + 1], 1);
        }
        S.sel[k] = sk;
    }
}

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
    const float upf = (float)up;
    const int64_t total = N * (int64_t)M;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += stride) {
        const int64_t i = q / M;
        const int j = (int)(q - i * M);
        const uint32_t wd = __ldg(x_bits + i * W + (j >> 5));
        grad_p[q] = ((wd >> (j & 31)) & 1u) ? upf : 0.f;
    }
}

__device__ __forceinline__ bool finite_nonneg(float v) { return v >= 0.f && v <= FLT_MAX; }

__global__ void validate_kernel(Params P, uint32_t *flags) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t bad = 0, maxb = 0;
    const int M = P.M, K = P.K;
    for (int64_t q = tid; q < P.N * M; q += stride)
        if (!finite_nonneg(P.p[q])) bad |= 1u;
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
    }
    for (int64_t k = tid; k < K; k += stride) {
        const double Bk = P.B[k];
        if (!(Bk > 0.0) || !(Bk < 1e300)) bad |= 16u;
    }
    if (bad) atomicOr(&flags[0], bad);
    if (maxb) atomicMax(&flags[1], maxb);
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

}  // namespace

cudaError_t launch_finalize(const Params &P, const Scratch &S, const double *lambda, double *R,
                            double *dual, double *primal, double *g, double alpha,
                            double *lambda_next, cudaStream_t st) {
    finalize_kernel<<<1, 256, 0, st>>>(P, S, lambda, R, dual, primal, g, alpha, lambda_next,
                                       lambda_next != nullptr);
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
    const int64_t total = P.N * (int64_t)P.M;
    int64_t blocks = (total + 255) / 256;
    const int64_t cap = (int64_t)sms * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    backward_kernel<<<(int)blocks, 256, 0, st>>>(P.N, P.M, P.W, P.K, lambda, x_bits, R, P.B, upstream,
                                                 grad_lambda, grad_p, grad_B);
    return cudaGetLastError();
}

cudaError_t launch_validate(const Params &P, uint32_t *flags, cudaStream_t st) {
    const int sms = sm_count();
    validate_kernel<<<sms * 4, 256, 0, st>>>(P, flags);
    return cudaGetLastError();
}

}  // namespace kp
