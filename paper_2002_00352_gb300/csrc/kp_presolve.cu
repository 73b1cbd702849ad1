// kp_presolve.cu -- pre-solving by sampling (Sec. 5.3): synchronous
// coordinate descent on a sample of n users, with every budget scaled by
// n / N, gives a starting lambda^0 for the whole instance (the paper reports
// 40-75 % fewer iterations from such a start).
//
// The sample is the caller's (a device list of user indices, so the random
// draw is an input); its rows are gathered into buffers of their own, a
// handle is created over them and kp_scd_step runs from lambda = 0.
#include <cstring>
#include <vector>

#include "kp_internal.h"

namespace {

constexpr int GATHER_THREADS = 256;

// sampled users' item rows (M values per user) of p, item counts, or dense b
// (M*K values per user); out-of-range user indices set *bad and copy nothing
template <typename T>
__global__ void gather_rows(const T *src, T *dst, const int64_t *users, int64_t n, int64_t N, int64_t row,
                            uint32_t *bad) {
    const int64_t total = n * row;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += stride) {
        const int64_t s = q / row, c = q - s * row;
        const int64_t u = users[s];
        if (u < 0 || u >= N) {
            *bad = 1u;
            continue;
        }
        dst[q] = src[u * row + c];
    }
}

// CSR: the number of entries of every sampled user
__global__ void csr_counts(const int64_t *uoff, const int64_t *users, int64_t n, int64_t N, int64_t *cnt,
                           uint32_t *bad) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += stride) {
        const int64_t u = users[s];
        if (u < 0 || u >= N) {
            *bad = 1u;
            cnt[s] = 0;
            continue;
        }
        cnt[s] = uoff[u + 1] - uoff[u];
    }
}

// CSR: one warp per sampled user copies its entries to their new place
__global__ void csr_gather_entries(const int64_t *uoff, const float *val, const int16_t *kidx,
                                   const int64_t *users, const int64_t *off2, int64_t n, int64_t N,
                                   float *val2, int16_t *kidx2) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < n; s += warps) {
        const int64_t u = users[s];
        if (u < 0 || u >= N) continue;  // reported by csr_counts
        const int64_t a = uoff[u], c = uoff[u + 1] - a, d = off2[s] - off2[0];
        for (int64_t e = lane; e < c; e += 32) {
            val2[d + e] = val[a + e];
            kidx2[d + e] = kidx[a + e];
        }
    }
}

__global__ void scale_budgets(const double *B, double f, double *B2, int K) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x) B2[k] = B[k] * f;
}

// the sample's buffers and handle, released together
struct Sample {
    std::vector<void *> mem;
    kp_problem *h = nullptr;
    template <typename T>
    cudaError_t alloc(T **p, size_t count) {
        void *q = nullptr;
        const cudaError_t e = cudaMalloc(&q, (count ? count : 1) * sizeof(T));
        if (e == cudaSuccess) mem.push_back(q);
        *p = (T *)q;
        return e;
    }
    ~Sample() {
        if (h) kp_destroy(h);
        for (void *q : mem) cudaFree(q);
    }
};

int grid_for(int64_t work) {
    int64_t g = (work + GATHER_THREADS - 1) / GATHER_THREADS;
    if (g > 4096) g = 4096;
    return g < 1 ? 1 : (int)g;
}

}  // namespace

extern "C" {

kp_status kp_presolve(kp_problem *h, const int64_t *users, int64_t n, int32_t iters, double *lambda0,
                      void *stream) {
    if (!h || !users || !lambda0) {
        kp::set_last_error("kp_presolve: NULL argument");
        return KP_EINVAL;
    }
    const kp::Params &P = h->P;
    if (n < 1 || n > P.N || iters < 0) {
        kp::set_last_error("kp_presolve: need 1 <= n <= N and iters >= 0");
        return KP_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int M = P.M, K = P.K;
    Sample smp;
    uint32_t *bad = nullptr;
    float *p2 = nullptr, *b2 = nullptr, *val2 = nullptr;
    uint8_t *nnz2 = nullptr;
    int16_t *kidx2 = nullptr;
    int64_t *off2 = nullptr, *cnt = nullptr;
    double *B2 = nullptr, *tmp = nullptr;
    cudaError_t e = cudaStreamSynchronize(st);  // the instance and lambda0 are ready
    if (e == cudaSuccess) e = smp.alloc(&bad, 1);
    if (e == cudaSuccess) e = cudaMemset(bad, 0, sizeof(uint32_t));
    if (e == cudaSuccess) e = smp.alloc(&p2, (size_t)n * M);
    if (e == cudaSuccess) e = smp.alloc(&B2, (size_t)K);
    if (e == cudaSuccess) e = smp.alloc(&tmp, (size_t)K);
    if (e == cudaSuccess) {
        gather_rows<float><<<grid_for(n * M), GATHER_THREADS>>>(P.p, p2, users, n, P.N, M, bad);
        scale_budgets<<<grid_for(K), GATHER_THREADS>>>(P.B, (double)n / (double)P.N, B2, K);
        e = cudaGetLastError();
    }
    int64_t nnz_total = 0;
    if (e == cudaSuccess && P.layout == KP_B_DENSE) {
        e = smp.alloc(&b2, (size_t)n * M * K);
        if (e == cudaSuccess) {
            gather_rows<float><<<grid_for(n * M * K), GATHER_THREADS>>>(P.b, b2, users, n, P.N, (int64_t)M * K, bad);
            e = cudaGetLastError();
        }
    } else if (e == cudaSuccess) {
        e = smp.alloc(&cnt, (size_t)n);
        if (e == cudaSuccess) e = smp.alloc(&off2, (size_t)n + 1);
        if (e == cudaSuccess) e = smp.alloc(&nnz2, (size_t)n * M);
        if (e == cudaSuccess) {
            csr_counts<<<grid_for(n), GATHER_THREADS>>>(P.uoff, users, n, P.N, cnt, bad);
            gather_rows<uint8_t><<<grid_for(n * M), GATHER_THREADS>>>(P.innz, nnz2, users, n, P.N, M, bad);
            e = cudaGetLastError();
        }
        // the sample's offsets: a prefix sum of n counts on the host
        std::vector<int64_t> hc, ho;
        if (e == cudaSuccess) {
            hc.resize((size_t)n);
            ho.resize((size_t)n + 1);
            e = cudaMemcpy(hc.data(), cnt, (size_t)n * sizeof(int64_t), cudaMemcpyDeviceToHost);
        }
        if (e == cudaSuccess) {
            ho[0] = 0;
            for (int64_t s = 0; s < n; ++s) ho[s + 1] = ho[s] + hc[s];
            nnz_total = ho[n];
            e = cudaMemcpy(off2, ho.data(), ((size_t)n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice);
        }
        if (e == cudaSuccess) e = smp.alloc(&val2, (size_t)nnz_total);
        if (e == cudaSuccess) e = smp.alloc(&kidx2, (size_t)nnz_total);
        if (e == cudaSuccess) {
            csr_gather_entries<<<grid_for(n * 32), GATHER_THREADS>>>(P.uoff, P.val, P.kidx, users, off2, n, P.N,
                                                                     val2, kidx2);
            e = cudaGetLastError();
        }
    }
    uint32_t hbad = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&hbad, bad, sizeof(hbad), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        kp::set_last_error(cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? KP_ENOMEM : KP_ECUDA;
    }
    if (hbad) {
        kp::set_last_error("kp_presolve: a sampled user index is outside 0..N-1");
        return KP_EINVAL;
    }
    // the sample as an instance of its own: the same local constraints
    std::vector<uint64_t> S((size_t)P.tree.L);
    std::vector<int32_t> Cc((size_t)P.tree.L);
    for (int l = 0; l < P.tree.L; ++l) {
        S[l] = P.tree.items[l];
        Cc[l] = P.tree.cap[l];
    }
    kp_desc d;
    memset(&d, 0, sizeof(d));
    d.N = n;
    d.M = M;
    d.K = K;
    d.p = p2;
    d.b_layout = P.layout;
    d.b_dense = b2;
    d.csr_user_off = off2;
    d.csr_item_nnz = nnz2;
    d.csr_val = val2;
    d.csr_k = kidx2;
    d.B = B2;
    d.L = P.tree.L;
    d.S = S.data();
    d.C = Cc.data();
    kp_status s = kp_create(&d, &smp.h);
    if (s != KP_OK) return s;
    // Algorithm 4 from lambda = 0 on the sample
    e = cudaMemsetAsync(lambda0, 0, (size_t)K * sizeof(double), st);
    if (e != cudaSuccess) {
        kp::set_last_error(cudaGetErrorString(e));
        return KP_ECUDA;
    }
    double *a = lambda0, *b = tmp;
    for (int t = 0; t < iters; ++t) {
        s = kp_scd_step(smp.h, a, b, nullptr, nullptr, nullptr, stream);
        if (s != KP_OK) return s;
        double *c = a;
        a = b;
        b = c;
    }
    if (a != lambda0) e = cudaMemcpyAsync(lambda0, a, (size_t)K * sizeof(double), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        kp::set_last_error(cudaGetErrorString(e));
        return KP_ECUDA;
    }
    return kp_device_status(smp.h, stream);
}

}  // extern "C"
