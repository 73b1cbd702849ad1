// kp_batch.cu -- many independent instances of the problem solved together:
// every pass over the users of all instances is one persistent launch over a
// work list of (instance, tile of users); the selection kernels run one block
// per (instance, knapsack).  Each instance keeps its own parameters, scratch,
// multipliers and counters; only the launches are shared.  An instance with
// enough tiles to fill the GPU several times over ("solo") gains nothing from
// sharing a launch: it runs its own passes, finalize and selection (the
// kernels of a single handle) inside the batched step, and the shared launches
// skip it.
#include <algorithm>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <vector>

#include "kp_internal.h"

struct kp_batch {
    int count = 0;
    std::vector<kp_problem *> probs;
    int maxm = 64;
    int G = 0;
    size_t smem[3] = {0, 0, 0};
    int64_t totK = 0, ntiles = 0;
    kp::BatchDev B{};
    kp::Counters *ctr = nullptr;
    uint32_t *bufcnt = nullptr;
    size_t bufcnt_words = 0;
    unsigned long long *next = nullptr;
    std::vector<void *> allocs;
    std::vector<int64_t> koff, xoff;
    std::vector<int> solo;  // instances that run their own launches
};

namespace {
// an instance with at least this many tiles per resident block runs solo
constexpr int SOLO_TILES_PER_BLOCK = 4;
}

namespace {

kp_status bfail(kp_status s, const char *msg, cudaError_t e = cudaSuccess) {
    char buf[320];
    if (e != cudaSuccess)
        snprintf(buf, sizeof(buf), "%s: %s", msg, cudaGetErrorString(e));
    else
        snprintf(buf, sizeof(buf), "%s", msg);
    kp::set_last_error(buf);
    return s;
}

template <class T>
kp_status bcopy(kp_batch *b, T **dst, const std::vector<T> &src, const char *what) {
    void *p = nullptr;
    const size_t bytes = std::max<size_t>(sizeof(T), src.size() * sizeof(T));
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) return bfail(KP_ENOMEM, what, e);
    b->allocs.push_back(p);
    if (!src.empty()) e = cudaMemcpy(p, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bfail(KP_ECUDA, what, e);
    *dst = static_cast<T *>(p);
    return KP_OK;
}

void destroy(kp_batch *b) {
    for (kp_problem *h : b->probs)
        if (h) kp_destroy(h);
    for (void *p : b->allocs) cudaFree(p);
    delete b;
}

int maxm_class(int M) { return M <= 8 ? 8 : (M <= 10 ? 10 : (M <= 16 ? 16 : 64)); }

}  // namespace

extern "C" {

kp_status kp_batch_create(const kp_desc *descs, int32_t count, kp_batch **out) {
    if (!descs || !out || count < 1) return bfail(KP_EINVAL, "kp_batch_create: NULL argument or count < 1");
    kp_batch *b = new (std::nothrow) kp_batch();
    if (!b) return bfail(KP_ENOMEM, "host allocation failed");
    b->count = count;
    b->probs.assign(count, nullptr);
    kp_status st = KP_OK;
    int maxM = 1;
    // parameters of every instance (validation and data scan as in kp_create)
    for (int i = 0; i < count && st == KP_OK; ++i) {
        if (descs[i].b_layout != KP_B_DENSE) {
            st = bfail(KP_EINVAL, "kp_batch_create: only dense instances can be batched");
            break;
        }
        b->probs[i] = new (std::nothrow) kp_problem();
        if (!b->probs[i]) {
            st = bfail(KP_ENOMEM, "host allocation failed");
            break;
        }
        st = kp_impl::prepare(&descs[i], b->probs[i]);
        maxM = std::max(maxM, (int)descs[i].M);
    }
    if (st != KP_OK) {
        destroy(b);
        return st;
    }
    b->maxm = maxm_class(maxM);
    for (int m = 0; m < 3; ++m)
        for (int i = 0; i < count; ++i) b->smem[m] = std::max(b->smem[m], kp::dense_smem_bytes(b->probs[i]->P, m));
    b->G = kp::batch_grid_size(b->maxm, b->smem[kp::MODE_HIST]);
    if (b->G < 1) {
        destroy(b);
        return bfail(KP_ECUDA, "kp_batch_create: no resident block fits the shared memory of the batch");
    }
    // estimated work of one user: the kinetic sweep per knapsack grows like M^3
    // (M lines, O(M^2) swaps, O(M) scan each); plus the reduced costs (M K)
    auto user_cost = [](const kp::Params &P) {
        const double m = (double)P.M;
        return (double)P.K * (m * m * (m + 8.0) / 8.0 + m + 16.0);
    };
    double total = 0.0;
    for (int i = 0; i < count; ++i) total += user_cost(b->probs[i]->P) * (double)b->probs[i]->P.N;
    // tiles of at most a quarter of a block's share of the work
    const double tile_target = total / (4.0 * b->G);
    for (int i = 0; i < count; ++i) {
        kp::Params &P = b->probs[i]->P;
        const double t = std::floor(tile_target / user_cost(P));
        if (t < (double)P.tile) P.tile = t < 1.0 ? 1 : (int)t;
    }
    for (int m = 0; m < 3; ++m) {
        b->smem[m] = 0;
        for (int i = 0; i < count; ++i) b->smem[m] = std::max(b->smem[m], kp::dense_smem_bytes(b->probs[i]->P, m));
    }
    // instances that fill the GPU on their own run solo; the work list holds
    // the tiles of every other instance, most expensive instances first
    std::vector<uint8_t> solo(count, 0);
    for (int i = 0; i < count; ++i) {
        const kp::Params &P = b->probs[i]->P;
        const int64_t tiles = (P.N + P.tile - 1) / P.tile;
        if (tiles >= (int64_t)SOLO_TILES_PER_BLOCK * b->G) {
            solo[i] = 1;
            b->solo.push_back(i);
            (void)kp::pass_grid_size(P);  // sets its kernels' attributes now, before any stream capture
        }
    }
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        return user_cost(b->probs[a]->P) > user_cost(b->probs[c]->P);
    });
    std::vector<int32_t> tile_inst;
    std::vector<int64_t> tile_u0, xoff(count);
    b->koff.assign(count + 1, 0);
    int64_t xo = 0;
    for (int i = 0; i < count; ++i) {
        const kp::Params &P = b->probs[i]->P;
        b->koff[i + 1] = b->koff[i] + P.K;
        xoff[i] = xo;
        xo += P.N * P.W;
    }
    for (int i : order) {
        if (solo[i]) continue;
        const kp::Params &P = b->probs[i]->P;
        for (int64_t u0 = 0; u0 < P.N; u0 += P.tile) {
            tile_inst.push_back(i);
            tile_u0.push_back(u0);
        }
    }
    b->ntiles = (int64_t)tile_inst.size();
    b->totK = b->koff[count];
    std::vector<int32_t> kinst(b->totK);
    for (int i = 0; i < count; ++i)
        for (int64_t k = b->koff[i]; k < b->koff[i + 1]; ++k) kinst[k] = i;
    {  // buffer counts of every instance in one array, cleared before each pass
        void *p = nullptr;
        b->bufcnt_words = (size_t)b->totK * b->G;
        cudaError_t e = cudaMalloc(&p, sizeof(uint32_t) * b->bufcnt_words);
        if (e == cudaSuccess) e = cudaMemset(p, 0, sizeof(uint32_t) * b->bufcnt_words);
        if (e != cudaSuccess) {
            destroy(b);
            return bfail(KP_ENOMEM, "batch buffer counts", e);
        }
        b->allocs.push_back(p);
        b->bufcnt = static_cast<uint32_t *>(p);
        e = cudaMalloc(&p, sizeof(unsigned long long) * (kp::MAX_REFINE + 1));
        if (e != cudaSuccess) {
            destroy(b);
            return bfail(KP_ENOMEM, "batch tile counters", e);
        }
        b->allocs.push_back(p);
        b->next = static_cast<unsigned long long *>(p);
    }
    {
        void *p = nullptr;
        cudaError_t e = cudaMalloc(&p, sizeof(kp::Counters) * count);
        if (e == cudaSuccess) e = cudaMemset(p, 0, sizeof(kp::Counters) * count);
        if (e != cudaSuccess) {
            destroy(b);
            return bfail(KP_ENOMEM, "batch counters", e);
        }
        b->allocs.push_back(p);
        b->ctr = static_cast<kp::Counters *>(p);
    }
    std::vector<kp::Params> hP(count);
    std::vector<kp::Scratch> hS(count);
    for (int i = 0; i < count && st == KP_OK; ++i) {
        kp_problem *h = b->probs[i];
        // the breakpoint buffer of a single handle (kp_create): a smaller one
        // overflows on large instances and costs re-run passes
        double budget = 4.0 * (double)h->P.N * h->P.M;
        budget = std::min(std::max(budget, (double)(1 << 20)), (double)(1 << 28));
        st = kp_impl::alloc_scratch(h, b->G, 0, b->G, budget, b->ctr + i,
                                    b->bufcnt + (size_t)b->koff[i] * b->G);
        hP[i] = h->P;
        hS[i] = h->S;
    }
    if (st == KP_OK) st = bcopy(b, const_cast<kp::Params **>(&b->B.P), hP, "batch parameters");
    if (st == KP_OK) st = bcopy(b, &b->B.S, hS, "batch scratch descriptors");
    if (st == KP_OK) st = bcopy(b, const_cast<int64_t **>(&b->B.koff), b->koff, "batch offsets");
    if (st == KP_OK) st = bcopy(b, const_cast<int64_t **>(&b->B.xoff), xoff, "batch x offsets");
    if (st == KP_OK) st = bcopy(b, const_cast<int32_t **>(&b->B.kinst), kinst, "batch knapsack table");
    if (st == KP_OK) st = bcopy(b, const_cast<uint8_t **>(&b->B.solo), solo, "batch solo flags");
    if (st == KP_OK) st = bcopy(b, const_cast<int32_t **>(&b->B.tile_inst), tile_inst, "batch tiles");
    if (st == KP_OK) st = bcopy(b, const_cast<int64_t **>(&b->B.tile_u0), tile_u0, "batch tiles");
    if (st != KP_OK) {
        destroy(b);
        return st;
    }
    b->xoff = xoff;
    b->B.ntiles = b->ntiles;
    b->B.count = count;
    b->B.next = b->next;
    *out = b;
    return KP_OK;
}

kp_status kp_batch_destroy(kp_batch *b) {
    if (!b) return KP_OK;
    cudaDeviceSynchronize();
    destroy(b);
    return KP_OK;
}

kp_status kp_batch_layout(kp_batch *b, int64_t *koff) {
    if (!b || !koff) return bfail(KP_EINVAL, "kp_batch_layout: NULL argument");
    for (int i = 0; i <= b->count; ++i) koff[i] = b->koff[i];
    return KP_OK;
}

// Clears the tile counters of a step and, for passes that buffer breakpoints,
// the buffer counts of every (instance, knapsack, block).
static cudaError_t reset_pass(kp_batch *b, bool counters, bool counts, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    if (counters) e = cudaMemsetAsync(b->next, 0, sizeof(unsigned long long) * (kp::MAX_REFINE + 1), st);
    if (e == cudaSuccess && counts) e = cudaMemsetAsync(b->bufcnt, 0, sizeof(uint32_t) * b->bufcnt_words, st);
    return e;
}

// The solo instances' share of a pass, finalize and selection: a single
// handle's launches on each instance's slice of the multipliers.
static cudaError_t solo_pass(kp_batch *b, const double *lam, int mode, int round, uint32_t *x_bits,
                             cudaStream_t st) {
    for (int i : b->solo) {
        const kp_problem *h = b->probs[i];
        cudaError_t e = kp::launch_user_pass(h->P, h->S, lam + b->koff[i], mode, round,
                                             x_bits ? x_bits + b->xoff[i] : nullptr, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

static cudaError_t solo_finalize(kp_batch *b, const double *lam, double *R, double *dual, double *primal,
                                 double alpha, double *lam_next, cudaStream_t st) {
    for (int i : b->solo) {
        const kp_problem *h = b->probs[i];
        const int64_t ko = b->koff[i];
        cudaError_t e = kp::launch_finalize(h->P, h->S, lam + ko, R ? R + ko : nullptr, dual ? dual + i : nullptr,
                                            primal ? primal + i : nullptr, nullptr, alpha,
                                            lam_next ? lam_next + ko : nullptr, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

static cudaError_t solo_select(kp_batch *b, const double *lam, double *lam_next, int round, cudaStream_t st) {
    for (int i : b->solo) {
        const kp_problem *h = b->probs[i];
        const int64_t ko = b->koff[i];
        cudaError_t e = kp::launch_select(h->P, h->S, lam + ko, lam_next + ko, round, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

kp_status kp_batch_reduce_consumption(kp_batch *b, const double *lambda, double *R, double *dual_sum,
                                      double *primal_sum, uint32_t *x_bits, void *stream) {
    if (!b || !lambda) return bfail(KP_EINVAL, "kp_batch_reduce_consumption: NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = reset_pass(b, true, false, st);
    if (e == cudaSuccess) e = kp::launch_batch_pass(b->B, b->maxm, b->smem[kp::MODE_STATE], b->G, lambda,
                                          kp::MODE_STATE, 0, x_bits, st);
    if (e == cudaSuccess) e = solo_pass(b, lambda, kp::MODE_STATE, 0, x_bits, st);
    if (e == cudaSuccess) e = kp::launch_batch_finalize(b->B, lambda, R, dual_sum, primal_sum, 0.0, nullptr, st);
    if (e == cudaSuccess) e = solo_finalize(b, lambda, R, dual_sum, primal_sum, 0.0, nullptr, st);
    if (e != cudaSuccess) return bfail(KP_ECUDA, "batch consumption pass", e);
    return KP_OK;
}

kp_status kp_batch_dd_step(kp_batch *b, const double *lambda, double alpha, double *lambda_next,
                           void *stream) {
    if (!b || !lambda || !lambda_next) return bfail(KP_EINVAL, "kp_batch_dd_step: NULL argument");
    if (!(alpha >= 0.0)) return bfail(KP_EINVAL, "kp_batch_dd_step: alpha must be >= 0");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = reset_pass(b, true, false, st);
    if (e == cudaSuccess)
        e = kp::launch_batch_pass(b->B, b->maxm, b->smem[kp::MODE_STATE], b->G, lambda, kp::MODE_STATE, 0,
                                  nullptr, st);
    if (e == cudaSuccess) e = solo_pass(b, lambda, kp::MODE_STATE, 0, nullptr, st);
    if (e == cudaSuccess) e = kp::launch_batch_finalize(b->B, lambda, nullptr, nullptr, nullptr, alpha, lambda_next, st);
    if (e == cudaSuccess) e = solo_finalize(b, lambda, nullptr, nullptr, nullptr, alpha, lambda_next, st);
    if (e != cudaSuccess) return bfail(KP_ECUDA, "batch dual-descent step", e);
    return KP_OK;
}

kp_status kp_batch_scd_step(kp_batch *b, const double *lambda, double *lambda_next, void *stream) {
    if (!b || !lambda || !lambda_next) return bfail(KP_EINVAL, "kp_batch_scd_step: NULL argument");
    if (lambda == lambda_next) return bfail(KP_EINVAL, "kp_batch_scd_step: lambda_next must not alias lambda");
    cudaStream_t st = (cudaStream_t)stream;
    // clear every instance's counters except its status word
    cudaError_t e = cudaMemset2DAsync(b->ctr, sizeof(kp::Counters), 0, offsetof(kp::Counters, status),
                                      (size_t)b->count, st);
    if (e == cudaSuccess) e = reset_pass(b, true, true, st);
    if (e == cudaSuccess)
        e = kp::launch_batch_pass(b->B, b->maxm, b->smem[kp::MODE_HIST], b->G, lambda, kp::MODE_HIST, 0,
                                  nullptr, st);
    if (e == cudaSuccess) e = solo_pass(b, lambda, kp::MODE_HIST, 0, nullptr, st);
    if (e == cudaSuccess) e = kp::launch_batch_finalize(b->B, lambda, nullptr, nullptr, nullptr, 0.0, nullptr, st);
    if (e == cudaSuccess) e = solo_finalize(b, lambda, nullptr, nullptr, nullptr, 0.0, nullptr, st);
    if (e == cudaSuccess) e = kp::launch_batch_select(b->B, b->totK, lambda, lambda_next, 0, st);
    if (e == cudaSuccess) e = solo_select(b, lambda, lambda_next, 0, st);
    for (int r = 1; r <= kp::MAX_REFINE && e == cudaSuccess; ++r) {
        e = reset_pass(b, false, true, st);
        if (e == cudaSuccess)
            e = kp::launch_batch_pass(b->B, b->maxm, b->smem[kp::MODE_REFINE], b->G, lambda, kp::MODE_REFINE, r,
                                  nullptr, st);
        if (e == cudaSuccess) e = solo_pass(b, lambda, kp::MODE_REFINE, r, nullptr, st);
        if (e == cudaSuccess) e = kp::launch_batch_select(b->B, b->totK, lambda, lambda_next, r, st);
        if (e == cudaSuccess) e = solo_select(b, lambda, lambda_next, r, st);
    }
    if (e != cudaSuccess) return bfail(KP_ECUDA, "batch SCD step", e);
    return KP_OK;
}

kp_status kp_batch_device_status(kp_batch *b, void *stream) {
    if (!b) return bfail(KP_EINVAL, "kp_batch_device_status: NULL batch");
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    std::vector<kp::Counters> h(b->count);
    if (e == cudaSuccess) e = cudaMemcpy(h.data(), b->ctr, sizeof(kp::Counters) * b->count, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return bfail(KP_ECUDA, "kp_batch_device_status", e);
    int32_t status = 0;
    for (const auto &c : h) status |= c.status;
    if (status) {
        e = cudaMemset2D(reinterpret_cast<char *>(b->ctr) + offsetof(kp::Counters, status), sizeof(kp::Counters), 0,
                         sizeof(int32_t), (size_t)b->count);
        if (e != cudaSuccess) return bfail(KP_ECUDA, "kp_batch_device_status", e);
    }
    if (status & (1 << KP_ETIMEOUT)) return bfail(KP_ETIMEOUT, "a kernel's bounded wait ran out");
    if (status & (1 << KP_ESTATE)) return bfail(KP_ESTATE, "threshold selection did not converge");
    return KP_OK;
}

}  // extern "C"
