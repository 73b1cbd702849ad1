// kp_internal.h -- structures shared by the host side of the C ABI and the
// kernels.  Not part of the public interface (include/kp.h is).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/kp.h"

namespace kp {

// Buckets of the per-knapsack breakpoint histogram built in the user pass.
// Sec. 5.2 buckets candidate lambda_k values by the logarithm of their
// distance from lambda_k^t.  Here the distance is measured in FP32 ulps
// (the bit patterns of positive floats are ordered like their values):
//   d = key(v1) - key(centre),  bucket = 32 + sign(d) (1 + floor(log2 |d|)),
// and bucket 32 holds d = 0.  64 buckets cover every positive float.
constexpr int NB = 64;
constexpr int NB_CENTRE = 32;
// sub-buckets used when a pass is re-run to narrow a key range
constexpr int NSUB = 256;
// re-run rounds of the user pass allowed inside one threshold selection
constexpr int MAX_REFINE = 4;
// smallest half-width (in buckets) of the buffered window around the centre
constexpr int WMIN = 12;

// per-knapsack state of the threshold selection (device resident)
struct SelK {
    uint32_t ckey;        // key of the bucket centre used by the last pass
    int32_t w;            // half-width of the buffered window for the next pass
    uint32_t lo, hi;      // unresolved key range [lo, hi)
    unsigned long long above;  // fixed-point mass strictly above hi
    int32_t state;        // 0 resolved, 1 needs a refine pass
    uint32_t last_nz_key; // key of the last non-zero lambda_k (centre when lambda_k = 0)
};

// global counters (device resident)
struct Counters {
    unsigned long long stats[3];  // passes used, resolved as zero, overflows
    int32_t n_unres[8];           // unresolved knapsacks after select round r
    int32_t status;               // bit kp_status set by a kernel (OR of causes)
};

// laminar tree of the local constraints, nodes in topological order
// (subsets first), so the lowest set bit of (path & mask) is the deepest node
struct Tree {
    int32_t L;
    uint32_t ipath[KP_MAX_M];  // bit l set iff item j belongs to node l
    uint8_t cap[KP_MAX_L];     // C_l clamped to 255
};

struct Params {
    int64_t N;
    int32_t M, K, layout, W;   // W = ceil(M/32) x words per user
    const float *p;
    const float *b;
    const int64_t *uoff;
    const uint8_t *innz;
    const float *val;
    const int16_t *kidx;
    const double *B;
    int32_t fixs;              // fixed-point shift: mass units of 2^-fixs
    Tree tree;
};

// device scratch owned by a handle
struct Scratch {
    int32_t G;                        // persistent grid size of the user pass
    int32_t cap_kb;                   // buffer entries per (k, block)
    unsigned long long *Rfix;         // [K]
    double *dual_part, *primal_part;  // [G]
    unsigned long long *hist;         // [K][NB]
    unsigned long long *subhist;      // [K][NSUB]
    uint2 *buf;                       // [K][G][cap_kb] (key, float bits of v2)
    uint32_t *bufcnt;                 // [K][G]
    uint32_t *ovf;                    // [K]
    SelK *sel;                        // [K]
    Counters *ctr;
};

enum PassMode { MODE_STATE = 0, MODE_HIST = 1, MODE_REFINE = 2 };

struct PassOut {
    uint32_t *x_bits;  // optional
};

// launchers (kp_pass.cu)
cudaError_t launch_user_pass(const Params &P, const Scratch &S, const double *lambda, int mode,
                             int round, uint32_t *x_bits, cudaStream_t st);
int pass_grid_size(const Params &P);
// launchers (kp_select.cu)
cudaError_t launch_finalize(const Params &P, const Scratch &S, const double *lambda, double *R,
                            double *dual, double *primal, double *g, double alpha,
                            double *lambda_next, cudaStream_t st);
cudaError_t launch_select(const Params &P, const Scratch &S, const double *lambda,
                          double *lambda_next, int round, cudaStream_t st);
cudaError_t launch_backward(const Params &P, const double *lambda, const uint32_t *x_bits,
                            const double *R, const double *upstream, double *grad_lambda,
                            float *grad_p, double *grad_B, cudaStream_t st);
cudaError_t launch_validate(const Params &P, uint32_t *flags, cudaStream_t st);

}  // namespace kp
