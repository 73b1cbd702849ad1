// kp_api.cu -- the extern "C" entry points declared in include/kp.h.
//
// Host-side validation of the instance description, creation of the
// handle's scratch memory, and the ordering of the kernel launches that make
// up one call.  No exception crosses the interface; errors are returned as
// kp_status with a thread-local message.
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "kp_internal.h"

namespace kp {
int pass_grid_size(const Params &P);
}


namespace {

thread_local char g_err[512] = "";

kp_status fail(kp_status s, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}

kp_status cuda_fail(cudaError_t e, const char *where) {
    return fail(e == cudaErrorMemoryAllocation ? KP_ENOMEM : KP_ECUDA, "%s: %s", where,
                cudaGetErrorString(e));
}

#define KP_CUDA(call, where)                          \
    do {                                              \
        cudaError_t e_ = (call);                      \
        if (e_ != cudaSuccess) return cuda_fail(e_, where); \
    } while (0)

template <class T>
kp_status alloc(kp_problem *h, T **out, size_t count, const char *what) {
    void *p = nullptr;
    size_t bytes = count * sizeof(T);
    if (bytes == 0) bytes = sizeof(T);
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) return fail(KP_ENOMEM, "cudaMalloc(%zu bytes) for %s: %s", bytes, what,
                                      cudaGetErrorString(e));
    h->allocs.push_back(p);
    e = cudaMemset(p, 0, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemset");
    *out = (T *)p;
    return KP_OK;
}

void free_all(kp_problem *h) {
    for (void *p : h->allocs) cudaFree(p);
    h->allocs.clear();
}

bool check_handle(kp_problem *h) { return h != nullptr && h->P.N > 0; }

}  // namespace

namespace kp {
// error text for kp_last_error() from entry points defined in other files
void set_last_error(const char *msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }
}  // namespace kp

extern "C" {

const char *kp_last_error(void) { return g_err; }

int kp_version(void) { return 100; }

}  // extern "C"

namespace kp_impl {

// Validates the description and fills P (host checks; the device scan of the
// instance into the caller's five flag words `flags`, on stream st, waited for;
// fixed-point shifts; CSR shape).  Allocates nothing.
kp_status fill_params(const kp_desc *d, kp::Params &P, uint32_t *flags, cudaStream_t st) {
    if (!d) return fail(KP_EINVAL, "NULL description");
    if (d->N < 1) return fail(KP_EINVAL, "N must be >= 1 (got %lld)", (long long)d->N);
    if (d->M < 1 || d->M > KP_MAX_M) return fail(KP_EINVAL, "M must be in 1..%d (got %d)", KP_MAX_M, d->M);
    if (d->K < 1 || d->K > KP_MAX_K) return fail(KP_EINVAL, "K must be in 1..%d (got %d)", KP_MAX_K, d->K);
    if (d->L < 0 || d->L > KP_MAX_L) return fail(KP_EINVAL, "L must be in 0..%d (got %d)", KP_MAX_L, d->L);
    if (!d->p || !d->B) return fail(KP_EINVAL, "p and B must be device pointers");
    if (d->b_layout == KP_B_DENSE) {
        if (!d->b_dense) return fail(KP_EINVAL, "dense layout needs b_dense");
    } else if (d->b_layout == KP_B_CSR) {
        if (!d->csr_user_off || !d->csr_item_nnz || !d->csr_val || !d->csr_k)
            return fail(KP_EINVAL, "CSR layout needs csr_user_off, csr_item_nnz, csr_val, csr_k");
    } else {
        return fail(KP_EINVAL, "unknown b_layout %d", d->b_layout);
    }
    if (d->L > 0 && (!d->S || !d->C)) return fail(KP_EINVAL, "S and C must be host arrays of length L");
    const uint64_t allm = d->M == 64 ? ~0ull : ((1ull << d->M) - 1);
    for (int l = 0; l < d->L; ++l) {
        if (d->S[l] == 0) return fail(KP_EINVAL, "local set %d is empty", l);
        if (d->S[l] & ~allm) return fail(KP_EINVAL, "local set %d names an item >= M", l);
        if (d->C[l] < 1) return fail(KP_EINVAL, "cap C_%d must be >= 1 (Sec. 2: C_l > 0)", l);
    }
    // Sec. 2.1, Definition 1
    for (int a = 0; a < d->L; ++a)
        for (int b = a + 1; b < d->L; ++b) {
            uint64_t i = d->S[a] & d->S[b];
            if (i != 0 && i != d->S[a] && i != d->S[b])
                return fail(KP_EINVAL, "local sets %d and %d are neither disjoint nor nested", a, b);
        }
    memset(&P, 0, sizeof(P));
    P.N = d->N;
    P.M = d->M;
    P.K = d->K;
    P.layout = d->b_layout;
    P.W = (d->M + 31) / 32;
    P.p = d->p;
    P.b = d->b_dense;
    P.uoff = d->csr_user_off;
    P.innz = d->csr_item_nnz;
    P.val = d->csr_val;
    P.kidx = d->csr_k;
    P.B = d->B;
    // topological order of the sets (subsets first: by size, ties by index)
    int order[KP_MAX_L];
    for (int l = 0; l < d->L; ++l) order[l] = l;
    for (int a = 1; a < d->L; ++a) {
        int v = order[a], b = a - 1;
        while (b >= 0 && __builtin_popcountll(d->S[order[b]]) > __builtin_popcountll(d->S[v])) {
            order[b + 1] = order[b];
            --b;
        }
        order[b + 1] = v;
    }
    P.tree.L = d->L;
    for (int t = 0; t < d->L; ++t) {
        int l = order[t];
        int c = d->C[l];
        P.tree.cap[t] = (uint8_t)(c > 255 ? 255 : c);
        P.tree.items[t] = d->S[l];
        for (int j = 0; j < d->M; ++j)
            if ((d->S[l] >> j) & 1ull) P.tree.ipath[j] |= 1u << t;
    }

    // device scan of the instance (Sec. 2 data assumptions); flags[3] starts at all ones
    cudaError_t e = cudaMemsetAsync(flags, 0, 5 * sizeof(uint32_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(flags + 3, 0xff, sizeof(uint32_t), st);
    if (e == cudaSuccess) e = kp::launch_validate(P, flags, st);
    uint32_t hf[5] = {0, 0, 0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "validate");
    if (hf[0])
        return fail(KP_EDATA, "instance violates Sec. 2 assumptions:%s%s%s%s%s",
                    (hf[0] & 1) ? " p negative or non-finite;" : "",
                    (hf[0] & 2) ? " b negative or non-finite;" : "",
                    (hf[0] & 4) ? " csr_user_off inconsistent with csr_item_nnz;" : "",
                    (hf[0] & 8) ? " csr_k out of range or not increasing within an item;" : "",
                    (hf[0] & 16) ? " B_k not positive and finite;" : "");
    float maxb;
    memcpy(&maxb, &hf[1], 4);
    if (!(maxb < 0x1p100f))  // breakpoints divide by b with the fast reciprocal
        return fail(KP_EDATA, "b values must be below 2^100 (max b = %g)", (double)maxb);
    double count;
    if (P.layout == KP_B_DENSE) {
        count = (double)P.N * P.M;
    } else {
        int64_t ends[2] = {0, 0};
        e = cudaMemcpyAsync(&ends[0], P.uoff, 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&ends[1], P.uoff + P.N, 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "csr offsets copy");
        count = (double)(ends[1] - ends[0]);
        P.uoff0 = ends[0];
        if (hf[3] == hf[4] && (hf[3] == 1 || hf[3] == 2)) {
            P.creg = (int)hf[3];
            const bool mexact = P.M == 8 || P.M == 10 || P.M == 16;
            const uintptr_t pp = (uintptr_t)P.p, vp = (uintptr_t)(P.val + P.uoff0),
                            kp2 = (uintptr_t)(P.kidx + P.uoff0);
            P.vec = mexact && (pp % 8 == 0) && (vp % 16 == 0) && (kp2 % 8 == 0) &&
                    ((P.M * P.creg) % 4 == 0);
        }
    }
    // fixed-point mass: every per-knapsack sum is below count * max b
    P.entries = count;
    P.maxb = maxb;
    P.fixs = kp::mass_shift(count, maxb);
    P.bscale = std::ldexp(1.0f, P.fixs);
    // objective sums: every per-user value is below M * max p
    float maxp;
    memcpy(&maxp, &hf[2], 4);
    P.maxp = maxp;
    double bo = (double)P.N * P.M * (double)maxp + 1.0;
    int so = (int)std::floor(62.0 - std::log2(bo));
    if (so > 40) so = 40;
    if (so < 0) so = 0;
    P.fixo = so;
    P.tile = P.layout == KP_B_DENSE ? kp::dense_tile_users(P) : 0;
    P.stage = 0;
    return KP_OK;
}

// Validates the description and fills h->P; the flag words of the scan are
// allocated for the call only.
kp_status prepare(const kp_desc *d, kp_problem *h) {
    int cur_dev = 0;
    KP_CUDA(cudaGetDevice(&cur_dev), "cudaGetDevice");
    h->device = cur_dev;
    uint32_t *flags = nullptr;
    cudaError_t ea = cudaMalloc(&flags, 5 * sizeof(uint32_t));
    if (ea != cudaSuccess) return fail(KP_ENOMEM, "cudaMalloc(validation flags): %s", cudaGetErrorString(ea));
    kp_status st = fill_params(d, h->P, flags, 0);
    cudaFree(flags);
    return st;
}

// Allocates the handle's scratch for blocks [g_lo, g_lo + gspan) of a grid of G
// blocks; budget = breakpoint-buffer entries; ctr, bufcnt = counters and
// buffer counts owned elsewhere (a batch pools them) or nullptr to allocate.
kp_status alloc_scratch(kp_problem *h, int G, int g_lo, int gspan, double budget,
                        kp::Counters *ctr, uint32_t *bufcnt) {
    kp_status st = KP_OK;
    const kp::Params &P = h->P;
    {
        kp::Scratch &S = h->S;
        S.G = G;
        S.g_lo = g_lo;
        // CSR: shared-entry masks, and the knapsacks three or more items of one
        // user use, which a kernel of their own sweeps into extra buffer blocks
        int rare_grid = 0;
        if (P.layout == KP_B_CSR) {
            unsigned long long *cnt = nullptr, n = 0;
            if ((st = alloc(h, &S.shmask, (size_t)P.N, "shared-entry masks")) != KP_OK) goto fail_out;
            if ((st = alloc(h, &cnt, 1, "rare-knapsack count")) != KP_OK) goto fail_out;
            cudaError_t e2 = kp::launch_shmask(P, S.shmask, nullptr, 0, cnt, 0);
            if (e2 == cudaSuccess) e2 = cudaMemcpy(&n, cnt, sizeof(n), cudaMemcpyDeviceToHost);
            if (e2 == cudaSuccess && n > 0) {
                unsigned long long *list = nullptr;
                if ((st = alloc(h, &list, (size_t)n, "rare-knapsack list")) != KP_OK) goto fail_out;
                e2 = cudaMemset(cnt, 0, sizeof(unsigned long long));
                if (e2 == cudaSuccess) e2 = kp::launch_shmask(P, S.shmask, list, (int64_t)n, cnt, 0);
                S.rare = list;
                S.nrare = (int64_t)n;
            }
            if (e2 == cudaSuccess) e2 = cudaDeviceSynchronize();
            if (e2 != cudaSuccess) {
                st = cuda_fail(e2, "shared-entry masks");
                goto fail_out;
            }
            if (S.nrare > 0) {
                int dev = 0, sms = 1;
                cudaGetDevice(&dev);
                cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
                // two resident blocks of 512 threads per SM (each owns buffer slots,
                // so few large blocks rather than many small ones)
                const long long want = (S.nrare + 511) / 512;
                rare_grid = (int)(want < 2 * sms ? want : 2 * sms);
            }
        }
        S.rare_blk0 = gspan;
        S.rare_grid = rare_grid;
        S.gspan = gspan + rare_grid;
        long long cap = (long long)(budget / ((double)P.K * S.gspan));
        if (cap < 64) cap = 64;
        S.cap_kb = (int)cap;
        const size_t K = (size_t)P.K, GS = (size_t)S.gspan;
        if ((st = alloc(h, &S.Rfix, K, "Rfix")) != KP_OK) goto fail_out;
        if ((st = alloc(h, &S.objfix, 2, "objective sums")) != KP_OK) goto fail_out;
        if ((st = alloc(h, &S.reg3, K * 3, "window masses")) != KP_OK) goto fail_out;
        if ((st = alloc(h, &S.subhist, K * kp::NSUB, "sub-histogram")) != KP_OK) goto fail_out;
        if ((st = alloc(h, &S.buf, K * GS * (size_t)S.cap_kb, "breakpoint buffer")) != KP_OK) goto fail_out;
        if (bufcnt)
            S.bufcnt = bufcnt;
        else if ((st = alloc(h, &S.bufcnt, K * GS, "buffer counts")) != KP_OK)
            goto fail_out;
        if ((st = alloc(h, &S.ovf, K, "overflow flags")) != KP_OK) goto fail_out;
        if ((st = alloc(h, &S.sel, K, "selection state")) != KP_OK) goto fail_out;
        if (ctr)
            S.ctr = ctr;
        else if ((st = alloc(h, &S.ctr, 1, "counters")) != KP_OK)
            goto fail_out;
        std::vector<kp::SelK> init(K);
        for (auto &x : init) {
            memset(&x, 0, sizeof(x));
            x.w = kp::WMIN_BITS;
        }
        cudaError_t e = cudaMemcpy(S.sel, init.data(), K * sizeof(kp::SelK), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            st = cuda_fail(e, "init selection state");
            goto fail_out;
        }
    }
fail_out:
    return st;
}

}  // namespace kp_impl

extern "C" {

kp_status kp_create(const kp_desc *d, kp_problem **out) {
    g_err[0] = 0;
    if (!d || !out) return fail(KP_EINVAL, "kp_create: NULL argument");
    kp_problem *h = new (std::nothrow) kp_problem();
    if (!h) return fail(KP_ENOMEM, "host allocation failed");
    kp_status st = kp_impl::prepare(d, h);
    if (st == KP_OK) {
        const char *env = getenv("KP_BUFFER_ENTRIES");
        double budget = env ? atof(env) : 4.0 * (double)h->P.N * h->P.M;
        if (!env) {
            if (budget < (double)(1 << 20)) budget = (double)(1 << 20);
            if (budget > (double)(1 << 28)) budget = (double)(1 << 28);
        }
        const int G = kp::pass_grid_size(h->P);
        st = kp_impl::alloc_scratch(h, G, 0, G, budget, nullptr);
    }
    if (st != KP_OK) {
        free_all(h);
        delete h;
        return st;
    }
    *out = h;
    return KP_OK;
}

kp_status kp_destroy(kp_problem *h) {
    if (!h) return KP_OK;
    cudaDeviceSynchronize();
    if (h->ppbuf) cudaFree(h->ppbuf);
    free_all(h);
    delete h;
    return KP_OK;
}

static kp_status state_pass(kp_problem *h, const double *lambda, uint32_t *x_bits, double *R,
                            double *dual, double *primal, double *g, double alpha,
                            double *lambda_next, cudaStream_t st) {
    cudaError_t e = kp::launch_user_pass(h->P, h->S, lambda, kp::MODE_STATE, 0, x_bits, st);
    if (e != cudaSuccess) return cuda_fail(e, "user pass");
    e = kp::launch_finalize(h->P, h->S, lambda, R, dual, primal, g, alpha, lambda_next, st);
    if (e != cudaSuccess) return cuda_fail(e, "finalize");
    return KP_OK;
}

kp_status kp_solve_users(kp_problem *h, const double *lambda, uint32_t *x_bits, void *stream) {
    if (!check_handle(h) || !lambda || !x_bits) return fail(KP_EINVAL, "kp_solve_users: NULL argument");
    return state_pass(h, lambda, x_bits, nullptr, nullptr, nullptr, nullptr, 0.0, nullptr,
                      (cudaStream_t)stream);
}

kp_status kp_reduce_consumption(kp_problem *h, const double *lambda, double *R, double *dual_sum,
                                double *primal_sum, double *g, uint32_t *x_bits, void *stream) {
    if (!check_handle(h) || !lambda) return fail(KP_EINVAL, "kp_reduce_consumption: NULL argument");
    return state_pass(h, lambda, x_bits, R, dual_sum, primal_sum, g, 0.0, nullptr,
                      (cudaStream_t)stream);
}

kp_status kp_dual_value(kp_problem *h, const double *lambda, double *g, void *stream) {
    if (!check_handle(h) || !lambda || !g) return fail(KP_EINVAL, "kp_dual_value: NULL argument");
    return state_pass(h, lambda, nullptr, nullptr, nullptr, nullptr, g, 0.0, nullptr,
                      (cudaStream_t)stream);
}

kp_status kp_dd_step(kp_problem *h, const double *lambda, double alpha, double *lambda_next,
                     double *R, void *stream) {
    if (!check_handle(h) || !lambda || !lambda_next) return fail(KP_EINVAL, "kp_dd_step: NULL argument");
    if (!(alpha >= 0.0)) return fail(KP_EINVAL, "kp_dd_step: alpha must be >= 0");
    return state_pass(h, lambda, nullptr, R, nullptr, nullptr, nullptr, alpha, lambda_next,
                      (cudaStream_t)stream);
}

kp_status kp_scd_breakpoints(kp_problem *h, const double *lambda, double *R, double *dual_sum,
                             double *primal_sum, uint32_t *x_bits, void *stream) {
    if (!check_handle(h) || !lambda) return fail(KP_EINVAL, "kp_scd_breakpoints: NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    KP_CUDA(cudaMemsetAsync(h->S.ctr, 0, offsetof(kp::Counters, status), st), "reset counters");
    cudaError_t e = kp::launch_user_pass(h->P, h->S, lambda, kp::MODE_HIST, 0, x_bits, st);
    if (e == cudaErrorInvalidConfiguration)
        return fail(KP_EINVAL, "kp_scd_breakpoints: the per-knapsack state of the breakpoint pass (K = %d) "
                               "does not fit in shared memory", h->P.K);
    if (e != cudaSuccess) return cuda_fail(e, "user pass (breakpoints)");
    e = kp::launch_finalize(h->P, h->S, lambda, R, dual_sum, primal_sum, nullptr, 0.0, nullptr, st);
    if (e != cudaSuccess) return cuda_fail(e, "finalize");
    return KP_OK;
}

kp_status kp_threshold_select(kp_problem *h, const double *lambda, double *lambda_next, void *stream) {
    if (!check_handle(h) || !lambda || !lambda_next) return fail(KP_EINVAL, "kp_threshold_select: NULL argument");
    if (lambda == lambda_next) return fail(KP_EINVAL, "kp_threshold_select: lambda_next must not alias lambda");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = kp::launch_select(h->P, h->S, lambda, lambda_next, 0, st);
    if (e != cudaSuccess) return cuda_fail(e, "select");
    for (int r = 1; r <= kp::MAX_REFINE; ++r) {
        e = kp::launch_user_pass(h->P, h->S, lambda, kp::MODE_REFINE, r, nullptr, st);
        if (e != cudaSuccess) return cuda_fail(e, "user pass (refine)");
        e = kp::launch_select(h->P, h->S, lambda, lambda_next, r, st);
        if (e != cudaSuccess) return cuda_fail(e, "select (refine)");
    }
    return KP_OK;
}

kp_status kp_scd_step(kp_problem *h, const double *lambda, double *lambda_next, double *R,
                      double *dual_sum, double *primal_sum, void *stream) {
    kp_status s = kp_scd_breakpoints(h, lambda, R, dual_sum, primal_sum, nullptr, stream);
    if (s != KP_OK) return s;
    return kp_threshold_select(h, lambda, lambda_next, stream);
}

kp_status kp_bcd_step(kp_problem *h, const double *lambda, const uint8_t *block, double *lambda_next,
                      double *dual_sum, double *primal_sum, void *stream) {
    if (!check_handle(h) || !lambda || !block || !lambda_next) return fail(KP_EINVAL, "kp_bcd_step: NULL argument");
    if (lambda == lambda_next) return fail(KP_EINVAL, "kp_bcd_step: lambda_next must not alias lambda");
    h->S.block = block;  // copied into every launch below
    kp_status s = kp_scd_breakpoints(h, lambda, nullptr, dual_sum, primal_sum, nullptr, stream);
    if (s == KP_OK) s = kp_threshold_select(h, lambda, lambda_next, stream);
    h->S.block = nullptr;
    return s;
}

kp_status kp_scd_step_bucketed(kp_problem *h, const double *lambda, double delta, double *lambda_next,
                               void *stream) {
    if (!check_handle(h) || !lambda || !lambda_next) return fail(KP_EINVAL, "kp_scd_step_bucketed: NULL argument");
    if (lambda == lambda_next) return fail(KP_EINVAL, "kp_scd_step_bucketed: lambda_next must not alias lambda");
    if (!(delta > 0.0) || !(delta <= 1e30)) return fail(KP_EINVAL, "kp_scd_step_bucketed: delta must be in (0, 1e30]");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = kp::launch_bucket_prep(h->P, h->S, lambda, delta, st);
    if (e == cudaSuccess)
        e = kp::launch_user_pass(h->P, h->S, lambda, kp::MODE_REFINE, kp::BUCKET_ROUND, nullptr, st);
    if (e == cudaSuccess) e = kp::launch_bucket_select(h->P, h->S, lambda, lambda_next, st);
    if (e != cudaSuccess) return cuda_fail(e, "kp_scd_step_bucketed");
    return KP_OK;
}

kp_status kp_dual_backward(kp_problem *h, const double *lambda, const uint32_t *x_bits,
                           const double *R, const double *upstream, double *grad_lambda,
                           float *grad_p, double *grad_B, void *stream) {
    if (!check_handle(h) || !lambda || !upstream) return fail(KP_EINVAL, "kp_dual_backward: NULL argument");
    if (grad_p && !x_bits) return fail(KP_EINVAL, "kp_dual_backward: grad_p needs x_bits");
    if (grad_lambda && !R) return fail(KP_EINVAL, "kp_dual_backward: grad_lambda needs R");
    cudaError_t e = kp::launch_backward(h->P, lambda, x_bits, R, upstream, grad_lambda, grad_p, grad_B,
                                        (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "backward");
    return KP_OK;
}

kp_status kp_autotune(kp_problem *h, int32_t *chosen, void *stream) {
    if (!check_handle(h)) return fail(KP_EINVAL, "kp_autotune: NULL handle");
    cudaStream_t st = (cudaStream_t)stream;
    kp::Params &P = h->P;
    if (P.layout != KP_B_DENSE) {  // the CSR pass has no run-time tile parameter
        if (chosen) *chosen = 0;
        return KP_OK;
    }
    // time the breakpoint pass on a prefix of the users at every candidate tile size
    kp::Params Q = P;
    Q.N = P.N < (1 << 18) ? P.N : (1 << 18);
    double *lam = nullptr;
    KP_CUDA(cudaMalloc(&lam, sizeof(double) * P.K), "cudaMalloc");
    KP_CUDA(cudaMemsetAsync(lam, 0, sizeof(double) * P.K, st), "cudaMemsetAsync");
    cudaEvent_t e0, e1;
    KP_CUDA(cudaEventCreate(&e0), "cudaEventCreate");
    KP_CUDA(cudaEventCreate(&e1), "cudaEventCreate");
    const int def = kp::dense_tile_users(P);
    int best = def, best_stage = 0;
    float best_ms = -1.f;
    const int cands[] = {def, 8, 16, 32, 64, 128, 256};
    for (int cs = 0; cs < 14; ++cs) {
        const int c = cands[cs % 7], stage = cs / 7;
        if (c > def && c != def) continue;  // larger tiles than the default do not fit its shared memory budget
        Q.tile = c;
        Q.stage = stage;
        cudaError_t e = kp::launch_user_pass(Q, h->S, lam, kp::MODE_HIST, 0, nullptr, st);  // warm
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        for (int r = 0; r < 3 && e == cudaSuccess; ++r)
            e = kp::launch_user_pass(Q, h->S, lam, kp::MODE_HIST, 0, nullptr, st);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            continue;
        }
        if (best_ms < 0.f || ms < best_ms) {
            best_ms = ms;
            best = c;
            best_stage = stage;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(lam);
    int32_t status = 0;  // a bounded wait that ran out while timing
    KP_CUDA(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    KP_CUDA(cudaMemcpy(&status, &h->S.ctr->status, 4, cudaMemcpyDeviceToHost), "status copy");
    // the timed passes accumulated into the scratch: clear what the next call consumes
    kp::Scratch &S = h->S;
    KP_CUDA(cudaMemsetAsync(S.Rfix, 0, sizeof(unsigned long long) * P.K, st), "cudaMemsetAsync");
    KP_CUDA(cudaMemsetAsync(S.objfix, 0, sizeof(unsigned long long) * 2, st), "cudaMemsetAsync");
    KP_CUDA(cudaMemsetAsync(S.reg3, 0, sizeof(unsigned long long) * 3 * P.K, st), "cudaMemsetAsync");
    KP_CUDA(cudaMemsetAsync(S.ovf, 0, sizeof(uint32_t) * P.K, st), "cudaMemsetAsync");
    KP_CUDA(cudaMemsetAsync(S.ctr, 0, sizeof(kp::Counters), st), "cudaMemsetAsync");
    KP_CUDA(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    if (status & (1 << KP_ETIMEOUT)) return fail(KP_ETIMEOUT, "kp_autotune: a timed pass's bounded wait ran out");
    P.tile = best;
    P.stage = best_stage;
    if (chosen) *chosen = best;
    return KP_OK;
}

kp_status kp_set_tile(kp_problem *h, int32_t users, int32_t staging) {
    if (!check_handle(h)) return fail(KP_EINVAL, "kp_set_tile: NULL handle");
    kp::Params &P = h->P;
    if (P.layout != KP_B_DENSE) return fail(KP_EINVAL, "kp_set_tile: the instance has no dense tiles");
    if (users == 0) users = kp::dense_tile_users(P);
    if (users < 1 || users > kp::dense_tile_users(P) || (staging != 0 && staging != 1))
        return fail(KP_EINVAL, "kp_set_tile: users must be in 1..%d and staging 0 or 1", kp::dense_tile_users(P));
    P.tile = users;
    P.stage = staging;
    return KP_OK;
}

kp_status kp_device_status(kp_problem *h, void *stream) {
    if (!check_handle(h)) return fail(KP_EINVAL, "kp_device_status: NULL handle");
    cudaStream_t st = (cudaStream_t)stream;
    KP_CUDA(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    int32_t status = 0;
    KP_CUDA(cudaMemcpy(&status, &h->S.ctr->status, 4, cudaMemcpyDeviceToHost), "status copy");
    KP_CUDA(cudaMemset(&h->S.ctr->status, 0, 4), "status reset");
    if (status & (1 << KP_ETIMEOUT)) return fail(KP_ETIMEOUT, "a kernel's bounded wait ran out");
    if (status & (1 << KP_ESTATE)) return fail(KP_ESTATE, "threshold selection did not converge");
    return KP_OK;
}

kp_status kp_info(kp_problem *h, int64_t out[4]) {
    if (!check_handle(h) || !out) return fail(KP_EINVAL, "kp_info: NULL argument");
    out[0] = h->S.G;
    out[1] = h->S.nrare;
    out[2] = h->S.rare_grid;
    out[3] = h->S.cap_kb;
    return KP_OK;
}

kp_status kp_wait_selftest(int64_t limit_ns, void *stream) {
    if (limit_ns < 1000 || limit_ns > 1000000000) return fail(KP_EINVAL, "kp_wait_selftest: limit_ns must be in [1e3, 1e9]");
    cudaStream_t st = (cudaStream_t)stream;
    int32_t *d = nullptr;
    KP_CUDA(cudaMalloc(&d, sizeof(int32_t)), "cudaMalloc");
    int32_t status = 0;
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(int32_t), st);
    if (e == cudaSuccess) e = kp::launch_wait_selftest((uint64_t)limit_ns, d, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&status, d, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(e, "kp_wait_selftest");
    if (status & (1 << KP_ETIMEOUT)) return fail(KP_ETIMEOUT, "kp_wait_selftest: the wait ran out (expected)");
    return KP_OK;
}

kp_status kp_limits(int32_t out[3]) {
    if (!out) return fail(KP_EINVAL, "kp_limits: NULL argument");
    out[0] = KP_MAX_M;
    out[1] = KP_MAX_L;
    out[2] = KP_MAX_K;
    return KP_OK;
}

kp_status kp_select_stats(kp_problem *h, int64_t out[3], void *stream) {
    if (!check_handle(h) || !out) return fail(KP_EINVAL, "kp_select_stats: NULL argument");
    KP_CUDA(cudaStreamSynchronize((cudaStream_t)stream), "cudaStreamSynchronize");
    unsigned long long s[3];
    KP_CUDA(cudaMemcpy(s, h->S.ctr->stats, sizeof(s), cudaMemcpyDeviceToHost), "stats copy");
    for (int q = 0; q < 3; ++q) out[q] = (int64_t)s[q];
    return KP_OK;
}

}  // extern "C"
