// kp_noalloc.cu -- kp_reduce_consumption_noalloc: the consumption pass of
// kp_reduce_consumption for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: a process whose device memory has
// been handed to its own pool (so an outside cudaMalloc fails or fragments
// that pool), or code on a latency-critical path that must not take the
// driver's allocation locks.  This entry point needs no handle: the few words
// of scratch the pass needs (per-knapsack fixed-point consumption sums, the
// two objective sums and the validation flags) live in one file-scope
// __device__ array of fixed size, so nothing is allocated on any call.
//
// The array is shared by every call on a device and keeps the last call's
// contents; each call clears what must start at zero.  Calls that overlap on
// the GPU (different streams, or different host threads) race on it.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "kp_internal.h"

namespace {

// Rfix [KP_MAX_K], objective sums [2], validation flags [5 x uint32 in 3 words]
constexpr int kScratchWords = KP_MAX_K + 2 + 3;
static __device__ __align__(256) unsigned long long g_scratch[kScratchWords];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned long long *g_ptr[kMaxDevices] = {};

kp_status fail(kp_status s, const char *msg, cudaError_t e = cudaSuccess) {
    char buf[256];
    if (e != cudaSuccess)
        snprintf(buf, sizeof(buf), "%s: %s", msg, cudaGetErrorString(e));
    else
        snprintf(buf, sizeof(buf), "%s", msg);
    kp::set_last_error(buf);
    return s;
}

// Device address of g_scratch on the current device, looked up once per device.
kp_status scratch_ptr(int dev, unsigned long long **out) {
    if (dev < 0 || dev >= kMaxDevices) return fail(KP_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return fail(KP_ECUDA, "cudaGetSymbolAddress", e);
        g_ptr[dev] = static_cast<unsigned long long *>(p);
    }
    *out = g_ptr[dev];
    return KP_OK;
}

}  // namespace

extern "C" {

kp_status kp_reduce_consumption_noalloc(const kp_desc *d, const double *lambda, double *R,
                                        double *dual_sum, double *primal_sum, double *g,
                                        uint32_t *x_bits, void *stream) {
    if (!d || !lambda) return fail(KP_EINVAL, "kp_reduce_consumption_noalloc: NULL argument");
    if (d->N < 1 || d->M < 1 || d->M > KP_MAX_M || d->L < 0 || d->L > KP_MAX_L)
        return fail(KP_EINVAL, "N, M or L out of range");
    if (d->K < 1 || d->K > KP_MAX_K)
        return fail(KP_EINVAL, "K out of range: this entry point's static scratch holds at most KP_MAX_K knapsacks");
    if (!d->p || !d->B) return fail(KP_EINVAL, "p and B must be device pointers");
    if (d->b_layout == KP_B_DENSE) {
        if (!d->b_dense) return fail(KP_EINVAL, "dense layout needs b_dense");
    } else if (d->b_layout == KP_B_CSR) {
        if (!d->csr_user_off || !d->csr_item_nnz || !d->csr_val || !d->csr_k)
            return fail(KP_EINVAL, "CSR layout needs csr_user_off, csr_item_nnz, csr_val, csr_k");
    } else {
        return fail(KP_EINVAL, "unknown b_layout");
    }
    if (d->L > 0 && (!d->S || !d->C)) return fail(KP_EINVAL, "S and C must be host arrays of length L");
    const uint64_t allm = d->M == 64 ? ~0ull : ((1ull << d->M) - 1);
    for (int l = 0; l < d->L; ++l)
        if (d->S[l] == 0 || (d->S[l] & ~allm) || d->C[l] < 1)
            return fail(KP_EINVAL, "empty local set, item >= M, or cap < 1");
    for (int a = 0; a < d->L; ++a)
        for (int b = a + 1; b < d->L; ++b) {
            const uint64_t i = d->S[a] & d->S[b];
            if (i != 0 && i != d->S[a] && i != d->S[b])
                return fail(KP_EINVAL, "local sets are neither disjoint nor nested (Sec. 2.1)");
        }
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(KP_ECUDA, "cudaGetDevice", e);
    unsigned long long *base = nullptr;
    kp_status s = scratch_ptr(dev, &base);
    if (s != KP_OK) return s;

    kp::Params P;
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
    int order[KP_MAX_L];
    for (int l = 0; l < d->L; ++l) order[l] = l;
    for (int a = 1; a < d->L; ++a) {  // subsets before supersets
        const int v = order[a];
        int b = a - 1;
        while (b >= 0 && __builtin_popcountll(d->S[order[b]]) > __builtin_popcountll(d->S[v])) {
            order[b + 1] = order[b];
            --b;
        }
        order[b + 1] = v;
    }
    P.tree.L = d->L;
    for (int t = 0; t < d->L; ++t) {
        const int l = order[t];
        P.tree.cap[t] = (uint8_t)(d->C[l] > 255 ? 255 : d->C[l]);
        P.tree.items[t] = d->S[l];
        for (int j = 0; j < d->M; ++j)
            if ((d->S[l] >> j) & 1ull) P.tree.ipath[j] |= 1u << t;
    }

    unsigned long long *Rfix = base;
    unsigned long long *objfix = base + KP_MAX_K;
    uint32_t *flags = reinterpret_cast<uint32_t *>(base + KP_MAX_K + 2);

    // clear the sums and flags left by the previous call; flags[3] starts at all ones
    e = cudaMemsetAsync(base, 0, sizeof(unsigned long long) * kScratchWords, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(flags + 3, 0xff, sizeof(uint32_t), st);
    if (e != cudaSuccess) return fail(KP_ECUDA, "cudaMemsetAsync", e);

    // the data scan of kp_create, into the static flags; read back synchronously
    e = kp::launch_validate(P, flags, st);
    uint32_t hf[5] = {0, 0, 0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(KP_ECUDA, "validation", e);
    if (hf[0]) return fail(KP_EDATA, "instance violates Sec. 2 assumptions (see kp_create)");
    float maxb, maxp;
    memcpy(&maxb, &hf[1], 4);
    memcpy(&maxp, &hf[2], 4);
    double count = (double)P.N * P.M;
    if (P.layout == KP_B_CSR) {
        int64_t ends[2] = {0, 0};
        e = cudaMemcpyAsync(&ends[0], P.uoff, 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&ends[1], P.uoff + P.N, 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return fail(KP_ECUDA, "csr offsets", e);
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
    P.fixs = kp::mass_shift(count, maxb);
    P.bscale = std::ldexp(1.0f, P.fixs);
    int fo = (int)std::floor(62.0 - std::log2((double)P.N * P.M * (double)maxp + 1.0));
    P.fixo = fo > 40 ? 40 : (fo < 0 ? 0 : fo);

    kp::Scratch S;
    memset(&S, 0, sizeof(S));
    S.G = kp::pass_grid_size(P);
    S.g_lo = 0;
    S.gspan = S.G;
    S.Rfix = Rfix;
    S.objfix = objfix;
    e = kp::launch_user_pass(P, S, lambda, kp::MODE_STATE, 0, x_bits, st);
    if (e == cudaSuccess) e = kp::launch_finalize(P, S, lambda, R, dual_sum, primal_sum, g, 0.0, nullptr, st);
    if (e != cudaSuccess) return fail(KP_ECUDA, "consumption pass", e);
    return KP_OK;
}

}  // extern "C"
