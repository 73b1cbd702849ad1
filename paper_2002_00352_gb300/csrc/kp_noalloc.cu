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
    if (d->K > KP_MAX_K)
        return fail(KP_EINVAL, "K out of range: this entry point's static scratch holds at most KP_MAX_K knapsacks");
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(KP_ECUDA, "cudaGetDevice", e);
    unsigned long long *base = nullptr;
    kp_status s = scratch_ptr(dev, &base);
    if (s != KP_OK) return s;
    unsigned long long *Rfix = base;
    unsigned long long *objfix = base + KP_MAX_K;
    uint32_t *flags = reinterpret_cast<uint32_t *>(base + KP_MAX_K + 2);

    // clear the sums left by the previous call
    e = cudaMemsetAsync(base, 0, sizeof(unsigned long long) * (KP_MAX_K + 2), st);
    if (e != cudaSuccess) return fail(KP_ECUDA, "cudaMemsetAsync", e);
    // the checks and the data scan of kp_create, into the static flag words
    kp::Params P;
    s = kp_impl::fill_params(d, P, flags, st);
    if (s != KP_OK) return s;

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
