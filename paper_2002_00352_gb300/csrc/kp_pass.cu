// kp_pass.cu -- the per-user pass of dual descent and synchronous coordinate
// descent (Algorithm 2 Map/Reduce, Algorithm 4 Map), one launch per pass over
// all users.
//
// Modes
//   MODE_STATE   reduced costs (Sec. 4.2), Algorithm 1 per user, x bits,
//                consumption R_k = sum_i v_ik (Algorithm 2), dual and primal
//                sums.
//   MODE_HIST    MODE_STATE + Algorithm 4's Map: every user's breakpoints of
//                its k-consumption, aggregated into per-knapsack histograms
//                bucketed around lambda_k^t (Sec. 5.2) plus a buffered window
//                of exact breakpoints around the centre.
//   MODE_REFINE  Algorithm 4's Map restricted to the key ranges still
//                unresolved by the threshold selection.
//
// Reductions: FP32 per user, exact 64-bit fixed point per knapsack (integer
// atomics, so the result does not depend on the order of the additions),
// FP64 per block for the objective sums and an ordered sum over blocks in
// the finalize kernel.  The grid is persistent and users are assigned to
// blocks statically, so every sum is reproducible run to run.
#include <cstdio>

#include "kp_device.cuh"
#include "kp_internal.h"

namespace kp {

namespace {

constexpr int HIST_SMEM_BYTES = 112 * 1024;   // per-block histogram kept in shared memory if it fits
constexpr int DENSE_TILE_BYTES = 64 * 1024;   // dense b tile

struct SmemLayout {
    size_t lamf, ckey, wwin, bcnt, lo, hi, shift, rfix, hist, rows, tile_p, tile_b, selm, red, total;
    bool hist_in_smem;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline SmemLayout smem_layout(int layout, int K, int M, int maxm, int threads,
                                                  int T, int mode) {
    SmemLayout s;
    size_t o = 0;
    s.lamf = o;
    o = align16(o + 4 * (size_t)K);
    s.ckey = o;
    o = align16(o + 4 * (size_t)K);
    s.wwin = o;
    o = align16(o + 4 * (size_t)K);
    s.bcnt = o;
    o = align16(o + 4 * (size_t)K);
    s.lo = o;
    o = align16(o + 4 * (size_t)K);
    s.hi = o;
    o = align16(o + 4 * (size_t)K);
    s.shift = o;
    o = align16(o + 4 * (size_t)K);
    s.rfix = o;
    o = align16(o + 8 * (size_t)K);
    s.hist_in_smem = (mode == MODE_HIST) && ((size_t)K * NB * 8 <= (size_t)HIST_SMEM_BYTES);
    s.hist = o;
    if (s.hist_in_smem) o = align16(o + (size_t)K * NB * 8);
    s.red = o;
    o = align16(o + 2 * 8 * 32);
    if (layout == KP_B_CSR) {
        s.rows = o;
        o = align16(o + 2 * 4 * (size_t)threads * maxm);
        s.tile_p = s.tile_b = s.selm = o;
    } else {
        s.tile_p = o;
        o = align16(o + 4 * (size_t)T * M);
        s.rows = o;  // p~ of the tile
        o = align16(o + 4 * (size_t)T * M);
        s.selm = o;
        o = align16(o + 8 * (size_t)T);
        s.tile_b = o;
        o = align16(o + 4 * (size_t)T * M * K);
    }
    s.total = o;
    return s;
}

__device__ __forceinline__ int bitlen(uint32_t x) { return x ? 32 - __clz(x) : 0; }

template <int MODE>
__device__ __forceinline__ void init_block_state(const Params &P, const Scratch &S,
                                                 const double *lam, const SmemLayout &L,
                                                 unsigned char *smem, int round) {
    const int K = P.K;
    float *lamf = (float *)(smem + L.lamf);
    uint32_t *ckey = (uint32_t *)(smem + L.ckey);
    int32_t *wwin = (int32_t *)(smem + L.wwin);
    uint32_t *bcnt = (uint32_t *)(smem + L.bcnt);
    uint32_t *lo = (uint32_t *)(smem + L.lo);
    uint32_t *hi = (uint32_t *)(smem + L.hi);
    int32_t *shift = (int32_t *)(smem + L.shift);
    unsigned long long *rfix = (unsigned long long *)(smem + L.rfix);
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        float lf = (float)lam[k];
        lamf[k] = lf;
        bcnt[k] = 0;
        rfix[k] = 0;
        if (MODE == MODE_HIST) {
            SelK sk = S.sel[k];
            uint32_t c = lf > 0.f ? __float_as_uint(lf) : sk.last_nz_key;
            ckey[k] = c;
            wwin[k] = sk.w;
            if (blockIdx.x == 0) S.sel[k].ckey = c;
        }
        if (MODE == MODE_REFINE) {
            SelK sk = S.sel[k];
            if (sk.state == 1) {
                lo[k] = sk.lo;
                hi[k] = sk.hi;
                uint32_t width = sk.hi - sk.lo;
                int sh = bitlen(width - 1) - 8;
                shift[k] = sh > 0 ? sh : 0;
            } else {
                lo[k] = 0;
                hi[k] = 0;
                shift[k] = 0;
            }
        }
    }
    if (MODE == MODE_HIST && L.hist_in_smem) {
        unsigned long long *h = (unsigned long long *)(smem + L.hist);
        for (int q = threadIdx.x; q < K * NB; q += blockDim.x) h[q] = 0ull;
    }
}

template <int MODE>
__device__ __forceinline__ void flush_block_state(const Params &P, const Scratch &S,
                                                  const SmemLayout &L, unsigned char *smem,
                                                  double dsum, double psum) {
    const int K = P.K;
    uint32_t *bcnt = (uint32_t *)(smem + L.bcnt);
    unsigned long long *rfix = (unsigned long long *)(smem + L.rfix);
    double *red = (double *)(smem + L.red);
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        if (MODE != MODE_REFINE && rfix[k]) atomicAdd(&S.Rfix[k], rfix[k]);
        if (MODE != MODE_STATE) {
            uint32_t c = bcnt[k];
            S.bufcnt[(size_t)k * S.G + blockIdx.x] = c < (uint32_t)S.cap_kb ? c : (uint32_t)S.cap_kb;
            if (c > (uint32_t)S.cap_kb) S.ovf[k] = 1u;
        }
    }
    if (MODE == MODE_HIST && L.hist_in_smem) {
        unsigned long long *h = (unsigned long long *)(smem + L.hist);
        for (int q = threadIdx.x; q < K * NB; q += blockDim.x)
            if (h[q]) atomicAdd(&S.hist[q], h[q]);
    }
    if (MODE != MODE_REFINE) {
        // block reduction of the FP64 objective sums in a fixed order
        for (int o = 16; o > 0; o >>= 1) {
            dsum += __shfl_down_sync(0xffffffffu, dsum, o);
            psum += __shfl_down_sync(0xffffffffu, psum, o);
        }
        int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (lane == 0) {
            red[wid] = dsum;
            red[32 + wid] = psum;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double a = 0.0, b = 0.0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
                a += red[q];
                b += red[32 + q];
            }
            S.dual_part[blockIdx.x] = a;
            S.primal_part[blockIdx.x] = b;
        }
    }
}

// ------------------------------------------------------------------------------------------
// CSR layout: one thread per user.
// ------------------------------------------------------------------------------------------
template <int MAXM, int MODE, class Sink>
__device__ __forceinline__ void csr_user(const Params &P, int64_t i, const float *lamf, float *pt,
                                         float *th, unsigned long long *rfix, double &dsum,
                                         double &psum, uint32_t *x_bits, Sink &sink) {
    const int M = P.M;
    const Tree &T = P.tree;
    const float *pr = P.p + (size_t)i * M;
    const uint8_t *nzr = P.innz + (size_t)i * M;
    const int64_t e0 = P.uoff[i];
    const float *val = P.val;
    const int16_t *kid = P.kidx;

    // Sec. 4.2: p~_ij = p_ij - sum_k lambda_k b_ijk over the item's entries
    uint64_t pos = 0;
    int64_t e = e0;
    for (int j = 0; j < M; ++j) {
        float acc = __ldg(pr + j);
        int c = nzr[j];
        for (int q = 0; q < c; ++q, ++e) acc = fmaf(-lamf[kid[e]], __ldg(val + e), acc);
        pt[j] = acc;
        if (acc > 0.f) pos |= 1ull << j;
    }
    // Algorithm 1
    Walk w;
    greedy_walk(pt, 1, pos, T, w);

    if (MODE != MODE_REFINE) {
        if (x_bits) {
            for (int q = 0; q < P.W; ++q) x_bits[(size_t)i * P.W + q] = (uint32_t)(w.sel >> (32 * q));
        }
        float scale = __uint_as_float((uint32_t)(127 + P.fixs) << 23);
        e = e0;
        for (int j = 0; j < M; ++j) {
            int c = nzr[j];
            if ((w.sel >> j) & 1ull) {
                dsum += (double)pt[j];
                psum += (double)__ldg(pr + j);
                for (int q = 0; q < c; ++q)
                    atomicAdd(&rfix[kid[e + q]], fixmass(__ldg(val + e + q), scale));
            }
            e += c;
        }
    }
    if (MODE != MODE_STATE) {
        item_thresholds(pt, M, w, T, th);
        e = e0;
        for (int j = 0; j < M; ++j) {
            int c = nzr[j];
            for (int q = 0; q < c; ++q) {
                const int64_t idx = e + q;
                const float v = __ldg(val + idx);
                if (!(v > 0.f)) continue;
                const int k = kid[idx];
                // does another item of this user also consume knapsack k?
                bool shared = false, first = true;
                int64_t f = e0;
                for (int j2 = 0; j2 < M; ++j2) {
                    int c2 = nzr[j2];
                    if (j2 != j) {
                        for (int q2 = 0; q2 < c2; ++q2)
                            if (kid[f + q2] == k && __ldg(val + f + q2) > 0.f) {
                                shared = true;
                                if (f + q2 < idx) first = false;
                            }
                    }
                    f += c2;
                }
                if (!shared) {
                    // single moving line: it is selected iff p~_j(lambda_k) > theta_j
                    float v1 = lamf[k] + (pt[j] - th[j]) / v;
                    sink.emit(k, v1, v);
                } else if (first) {
                    float s[MAXM];
                    uint64_t J = 0;
                    int64_t f2 = e0;
                    for (int j2 = 0; j2 < M; ++j2) {
                        int c2 = nzr[j2];
                        s[j2] = 0.f;
                        for (int q2 = 0; q2 < c2; ++q2)
                            if (kid[f2 + q2] == k) {
                                float vv = __ldg(val + f2 + q2);
                                if (vv > 0.f) {
                                    s[j2] = vv;
                                    J |= 1ull << j2;
                                }
                            }
                        f2 += c2;
                    }
                    sweep_k<MAXM>(pt, 1, s, 1, M, J, lamf[k], T, k, sink);
                }
            }
            e += c;
        }
    }
}

template <int MAXM, int MODE, int THREADS>
__global__ void __launch_bounds__(THREADS) csr_pass_kernel(Params P, Scratch S, const double *lam,
                                                           uint32_t *x_bits, int round) {
    extern __shared__ __align__(16) unsigned char smem[];
    if (MODE == MODE_REFINE && S.ctr->n_unres[round] == 0) return;
    if (MODE != MODE_STATE && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&S.ctr->stats[0], 1ull);
    const SmemLayout L = smem_layout(KP_B_CSR, P.K, P.M, MAXM, THREADS, 0, MODE);
    init_block_state<MODE>(P, S, lam, L, smem, round);
    __syncthreads();
    const float *lamf = (const float *)(smem + L.lamf);
    unsigned long long *rfix = (unsigned long long *)(smem + L.rfix);
    float *pt = (float *)(smem + L.rows) + (size_t)threadIdx.x * MAXM;
    float *th = (float *)(smem + L.rows) + (size_t)(THREADS + threadIdx.x) * MAXM;
    double dsum = 0.0, psum = 0.0;

    HistSink hs;
    RefineSink rs;
    if (MODE == MODE_HIST) {
        hs.hist = L.hist_in_smem ? (unsigned long long *)(smem + L.hist) : S.hist;
        hs.ckey = (const uint32_t *)(smem + L.ckey);
        hs.wwin = (const int32_t *)(smem + L.wwin);
        hs.bcnt = (uint32_t *)(smem + L.bcnt);
        hs.buf = S.buf;
        hs.cap_kb = S.cap_kb;
        hs.G = S.G;
        hs.blk = blockIdx.x;
        hs.scale = __uint_as_float((uint32_t)(127 + P.fixs) << 23);
    }
    if (MODE == MODE_REFINE) {
        rs.lo = (const uint32_t *)(smem + L.lo);
        rs.hi = (const uint32_t *)(smem + L.hi);
        rs.shift = (const int32_t *)(smem + L.shift);
        rs.subhist = S.subhist;
        rs.bcnt = (uint32_t *)(smem + L.bcnt);
        rs.buf = S.buf;
        rs.cap_kb = S.cap_kb;
        rs.G = S.G;
        rs.blk = blockIdx.x;
        rs.scale = __uint_as_float((uint32_t)(127 + P.fixs) << 23);
    }
    const int64_t stride = (int64_t)gridDim.x * THREADS;
    for (int64_t i = (int64_t)blockIdx.x * THREADS + threadIdx.x; i < P.N; i += stride) {
        if (MODE == MODE_HIST)
            csr_user<MAXM, MODE>(P, i, lamf, pt, th, rfix, dsum, psum, x_bits, hs);
        else if (MODE == MODE_REFINE)
            csr_user<MAXM, MODE>(P, i, lamf, pt, th, rfix, dsum, psum, x_bits, rs);
        else {
            NullSink ns;
            csr_user<MAXM, MODE>(P, i, lamf, pt, th, rfix, dsum, psum, x_bits, ns);
        }
    }
    flush_block_state<MODE>(P, S, L, smem, dsum, psum);
}

// ------------------------------------------------------------------------------------------
// Dense layout: a tile of T users is staged in shared memory; reduced costs are
// computed per (user, item), the greedy per user, and consumption and the
// breakpoints per (user, knapsack).
// ------------------------------------------------------------------------------------------
template <int MAXM, int MODE, int THREADS>
__global__ void __launch_bounds__(THREADS) dense_pass_kernel(Params P, Scratch S, const double *lam,
                                                             uint32_t *x_bits, int round, int T) {
    extern __shared__ __align__(16) unsigned char smem[];
    if (MODE == MODE_REFINE && S.ctr->n_unres[round] == 0) return;
    if (MODE != MODE_STATE && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&S.ctr->stats[0], 1ull);
    const int M = P.M, K = P.K;
    const SmemLayout L = smem_layout(KP_B_DENSE, K, M, MAXM, THREADS, T, MODE);
    init_block_state<MODE>(P, S, lam, L, smem, round);
    __syncthreads();
    const float *lamf = (const float *)(smem + L.lamf);
    unsigned long long *rfix = (unsigned long long *)(smem + L.rfix);
    float *tp = (float *)(smem + L.tile_p);
    float *tb = (float *)(smem + L.tile_b);
    float *pt = (float *)(smem + L.rows);
    uint64_t *selm = (uint64_t *)(smem + L.selm);
    const float scale = __uint_as_float((uint32_t)(127 + P.fixs) << 23);
    double dsum = 0.0, psum = 0.0;

    HistSink hs;
    RefineSink rs;
    if (MODE == MODE_HIST) {
        hs.hist = L.hist_in_smem ? (unsigned long long *)(smem + L.hist) : S.hist;
        hs.ckey = (const uint32_t *)(smem + L.ckey);
        hs.wwin = (const int32_t *)(smem + L.wwin);
        hs.bcnt = (uint32_t *)(smem + L.bcnt);
        hs.buf = S.buf;
        hs.cap_kb = S.cap_kb;
        hs.G = S.G;
        hs.blk = blockIdx.x;
        hs.scale = scale;
    }
    if (MODE == MODE_REFINE) {
        rs.lo = (const uint32_t *)(smem + L.lo);
        rs.hi = (const uint32_t *)(smem + L.hi);
        rs.shift = (const int32_t *)(smem + L.shift);
        rs.subhist = S.subhist;
        rs.bcnt = (uint32_t *)(smem + L.bcnt);
        rs.buf = S.buf;
        rs.cap_kb = S.cap_kb;
        rs.G = S.G;
        rs.blk = blockIdx.x;
        rs.scale = scale;
    }
    const bool b_al = ((reinterpret_cast<uintptr_t>(P.b) & 15u) == 0) && ((M * K) % 4 == 0 || T % 4 == 0);
    const bool p_al = ((reinterpret_cast<uintptr_t>(P.p) & 15u) == 0) && ((M % 4) == 0 || T % 4 == 0);
    const int64_t ntiles = (P.N + T - 1) / T;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t u0 = tile * T;
        const int nu = (int)((P.N - u0) < T ? (P.N - u0) : T);
        // stage the tile
        {
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
        __syncthreads();
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
                while (r) {
                    int j = __ffsll((long long)r) - 1;
                    r &= r - 1;
                    dsum += (double)ptu[j];
                    psum += (double)tp[(size_t)u * M + j];
                }
            }
        }
        __syncthreads();
        // per (user, knapsack): consumption and Algorithm 4's Map
        for (int idx = threadIdx.x; idx < nu * K; idx += THREADS) {
            const int u = idx / K, k = idx - u * K;
            const float *bcol = tb + (size_t)u * M * K + k;
            if (MODE != MODE_REFINE) {
                uint64_t r = selm[u];
                unsigned long long acc = 0ull;
                while (r) {
                    int j = __ffsll((long long)r) - 1;
                    r &= r - 1;
                    acc += fixmass(bcol[(size_t)j * K], scale);
                }
                if (acc) atomicAdd(&rfix[k], acc);
            }
            if (MODE != MODE_STATE) {
                uint64_t J = 0;
                for (int j = 0; j < M; ++j)
                    if (bcol[(size_t)j * K] > 0.f) J |= 1ull << j;
                if (MODE == MODE_HIST)
                    sweep_k<MAXM>(pt + (size_t)u * M, 1, bcol, K, M, J, lamf[k], P.tree, k, hs);
                else
                    sweep_k<MAXM>(pt + (size_t)u * M, 1, bcol, K, M, J, lamf[k], P.tree, k, rs);
            }
        }
        __syncthreads();
    }
    flush_block_state<MODE>(P, S, L, smem, dsum, psum);
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

constexpr int CSR_THREADS = 256;
constexpr int DENSE_THREADS = 256;

int dense_tile_users(const Params &P) {
    long long per = (long long)P.M * P.K * 4;
    long long T = DENSE_TILE_BYTES / per;
    if (T > 256) T = 256;
    if (T >= 4) T &= ~3LL;
    if (T < 1) T = 1;
    return (int)T;
}

template <int MAXM, int MODE>
cudaError_t launch_t(const Params &P, const Scratch &S, const double *lam, uint32_t *x_bits,
                     int round, cudaStream_t st, int *occupancy_out) {
    if (P.layout == KP_B_CSR) {
        SmemLayout L = smem_layout(KP_B_CSR, P.K, P.M, MAXM, CSR_THREADS, 0, MODE);
        auto kern = csr_pass_kernel<MAXM, MODE, CSR_THREADS>;
        static bool attr_done = false;  // once per instantiation, before any stream capture
        if (!attr_done) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, max_optin_smem());
            if (e != cudaSuccess) return e;
            attr_done = true;
        }
        if (L.total > (size_t)max_optin_smem()) return cudaErrorInvalidConfiguration;
        if (occupancy_out) {
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occupancy_out, kern, CSR_THREADS, L.total);
        }
        kern<<<S.G, CSR_THREADS, L.total, st>>>(P, S, lam, x_bits, round);
        return cudaGetLastError();
    } else {
        int T = dense_tile_users(P);
        SmemLayout L = smem_layout(KP_B_DENSE, P.K, P.M, MAXM, DENSE_THREADS, T, MODE);
        auto kern = dense_pass_kernel<MAXM, MODE, DENSE_THREADS>;
        static bool attr_done = false;  // once per instantiation, before any stream capture
        if (!attr_done) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, max_optin_smem());
            if (e != cudaSuccess) return e;
            attr_done = true;
        }
        if (L.total > (size_t)max_optin_smem()) return cudaErrorInvalidConfiguration;
        if (occupancy_out) {
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occupancy_out, kern, DENSE_THREADS, L.total);
        }
        kern<<<S.G, DENSE_THREADS, L.total, st>>>(P, S, lam, x_bits, round, T);
        return cudaGetLastError();
    }
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
    if (P.M <= 16) return launch_m<16>(P, S, lam, mode, round, x_bits, st, occ);
    return launch_m<64>(P, S, lam, mode, round, x_bits, st, occ);
}

}  // namespace

cudaError_t launch_user_pass(const Params &P, const Scratch &S, const double *lambda, int mode,
                             int round, uint32_t *x_bits, cudaStream_t st) {
    return dispatch(P, S, lambda, mode, round, x_bits, st, nullptr);
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
    if (occ > 4) occ = 4;
    return sms * occ;
}

size_t pass_smem_bytes(const Params &P, int mode) {
    int maxm = P.M <= 16 ? 16 : 64;
    if (P.layout == KP_B_CSR) return smem_layout(KP_B_CSR, P.K, P.M, maxm, CSR_THREADS, 0, mode).total;
    return smem_layout(KP_B_DENSE, P.K, P.M, maxm, DENSE_THREADS, dense_tile_users(P), mode).total;
}

}  // namespace kp
