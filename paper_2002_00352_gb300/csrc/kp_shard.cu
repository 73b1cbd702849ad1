// kp_shard.cu -- one instance whose users are split over several handles
// ("shards", e.g. one per GPU), solved as one: users are independent given
// lambda (Sec. 4.1), so every shard runs the user passes of its own users, and
// the Reduce of Algorithm 4 (and Algorithm 2's sums) combines the shards'
// integer partials (fixed-point consumption and objective sums, window masses,
// sub-histograms) and their buffered breakpoints.  The lead shard's finalize
// and selection kernels read the other shards' scratch through a device array
// of their descriptors; all shards share one fixed-point unit, so every sum is
// exact and the result equals that of one handle over all the users.
//
// The shards must live on the device that is current at every call (the
// kernels read the other shards' memory directly).
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <vector>

#include "kp_internal.h"

struct kp_shard_group {
    std::vector<kp_problem *> shards;
    kp::Scratch *dpeers = nullptr;  // [n - 1] device copies of the other shards' descriptors
};

namespace {

kp_status sfail(kp_status s, const char *msg, cudaError_t e = cudaSuccess) {
    char buf[320];
    if (e != cudaSuccess)
        snprintf(buf, sizeof(buf), "%s: %s", msg, cudaGetErrorString(e));
    else
        snprintf(buf, sizeof(buf), "%s", msg);
    kp::set_last_error(buf);
    return s;
}

bool same_tree(const kp::Tree &a, const kp::Tree &b, int M) {
    if (a.L != b.L) return false;
    for (int l = 0; l < a.L; ++l)
        if (a.items[l] != b.items[l] || a.cap[l] != b.cap[l]) return false;
    for (int j = 0; j < M; ++j)
        if (a.ipath[j] != b.ipath[j]) return false;
    return true;
}

}  // namespace

extern "C" {

kp_status kp_shard_group_create(kp_problem *const *shards, int32_t n, kp_shard_group **out) {
    if (!shards || !out || n < 1) return sfail(KP_EINVAL, "kp_shard_group_create: NULL argument or n < 1");
    const kp_problem *lead = shards[0];
    for (int r = 0; r < n; ++r) {
        const kp_problem *h = shards[r];
        if (!h || h->P.N < 1) return sfail(KP_EINVAL, "kp_shard_group_create: NULL shard");
        if (h->device != lead->device || h->P.K != lead->P.K || h->P.M != lead->P.M ||
            h->P.layout != lead->P.layout || !same_tree(h->P.tree, lead->P.tree, h->P.M))
            return sfail(KP_EINVAL, "kp_shard_group_create: shards differ in device, K, M, layout or local sets");
        for (int q = 0; q < r; ++q)
            if (shards[q] == h) return sfail(KP_EINVAL, "kp_shard_group_create: a handle appears twice");
    }
    // one fixed-point unit for all shards: the one a single handle over all the
    // users would choose
    double entries = 0.0, users = 0.0;
    float maxb = 0.f, maxp = 0.f;
    for (int r = 0; r < n; ++r) {
        entries += shards[r]->P.entries;
        users += (double)shards[r]->P.N;
        maxb = std::fmax(maxb, shards[r]->P.maxb);
        maxp = std::fmax(maxp, shards[r]->P.maxp);
    }
    const int fixs = kp::mass_shift(entries, maxb);
    int fixo = (int)std::floor(62.0 - std::log2(users * lead->P.M * (double)maxp + 1.0));
    fixo = fixo > 40 ? 40 : (fixo < 0 ? 0 : fixo);
    kp_shard_group *g = new (std::nothrow) kp_shard_group();
    if (!g) return sfail(KP_ENOMEM, "host allocation failed");
    for (int r = 0; r < n; ++r) {
        shards[r]->P.fixs = fixs;
        shards[r]->P.bscale = std::ldexp(1.0f, fixs);
        shards[r]->P.fixo = fixo;
        g->shards.push_back(shards[r]);
    }
    if (n > 1) {
        std::vector<kp::Scratch> hp;
        for (int r = 1; r < n; ++r) hp.push_back(shards[r]->S);
        cudaError_t e = cudaMalloc(&g->dpeers, sizeof(kp::Scratch) * hp.size());
        if (e == cudaSuccess) e = cudaMemcpy(g->dpeers, hp.data(), sizeof(kp::Scratch) * hp.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(g->dpeers);
            delete g;
            return sfail(KP_ENOMEM, "kp_shard_group_create: peer descriptors", e);
        }
    }
    *out = g;
    return KP_OK;
}

kp_status kp_shard_group_destroy(kp_shard_group *g) {
    if (!g) return KP_OK;
    cudaDeviceSynchronize();
    cudaFree(g->dpeers);
    delete g;
    return KP_OK;
}

kp_status kp_shard_group_scd_step(kp_shard_group *g, const double *lambda, double *lambda_next, double *R,
                                  double *dual_sum, double *primal_sum, void *stream) {
    if (!g || !lambda || !lambda_next) return sfail(KP_EINVAL, "kp_shard_group_scd_step: NULL argument");
    if (lambda == lambda_next) return sfail(KP_EINVAL, "kp_shard_group_scd_step: lambda_next must not alias lambda");
    cudaStream_t st = (cudaStream_t)stream;
    kp_problem *lead = g->shards[0];
    const int n = (int)g->shards.size();
    const size_t selb = sizeof(kp::SelK) * (size_t)lead->P.K;
    // every shard works from the lead's selection state (window, ranges); the
    // other shards' re-run passes read the lead's counters of unresolved knapsacks
    auto sync_state = [&]() -> cudaError_t {
        for (int r = 1; r < n; ++r) {
            cudaError_t e = cudaMemcpyAsync(g->shards[r]->S.sel, lead->S.sel, selb, cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    };
    auto shard_scratch = [&](int r) {
        kp::Scratch S = g->shards[r]->S;
        S.ctr = lead->S.ctr;
        return S;
    };
    kp::Scratch SL = lead->S;  // the lead's selection reads the other shards' partials
    SL.peers = g->dpeers;
    SL.npeers = n - 1;
    cudaError_t e = sync_state();
    if (e == cudaSuccess) e = cudaMemsetAsync(lead->S.ctr, 0, offsetof(kp::Counters, status), st);
    for (int r = 0; r < n && e == cudaSuccess; ++r)
        e = kp::launch_user_pass(g->shards[r]->P, shard_scratch(r), lambda, kp::MODE_HIST, 0, nullptr, st);
    if (e == cudaSuccess)
        e = kp::launch_finalize(lead->P, SL, lambda, R, dual_sum, primal_sum, nullptr, 0.0, nullptr, st);
    if (e == cudaSuccess) e = kp::launch_select(lead->P, SL, lambda, lambda_next, 0, st);
    for (int round = 1; round <= kp::MAX_REFINE && e == cudaSuccess; ++round) {
        e = sync_state();
        for (int r = 0; r < n && e == cudaSuccess; ++r)
            e = kp::launch_user_pass(g->shards[r]->P, shard_scratch(r), lambda, kp::MODE_REFINE, round, nullptr, st);
        if (e == cudaSuccess) e = kp::launch_select(lead->P, SL, lambda, lambda_next, round, st);
    }
    if (e == cudaSuccess) e = sync_state();
    if (e != cudaSuccess) return sfail(KP_ECUDA, "kp_shard_group_scd_step", e);
    return KP_OK;
}

}  // extern "C"
