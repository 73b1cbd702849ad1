// kp_internal.h -- structures shared by the host side of the C ABI and the
// kernels.  Not part of the public interface (include/kp.h is).
#pragma once
#include <cmath>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/kp.h"

namespace kp {

// Threshold selection (Reduce of Algorithm 4).  The breakpoint pass splits
// every knapsack's breakpoints into three key ranges around a predicted
// threshold (Sec. 5.2 centres its buckets at lambda_k^t for the same reason):
// above the window, inside it and below it.  The masses of the three ranges
// are accumulated exactly (64-bit fixed point) and the breakpoints inside the
// window are buffered, so when the crossing falls inside the window the exact
// breakpoint is selected from the buffer; otherwise the pass is re-run over the
// range that holds the crossing with a 256-way sub-histogram.  Keys are the
// FP32 bit patterns of the breakpoints, ordered like their values.
constexpr uint32_t KEY_INF = 0x7F800000u;
// sub-buckets used when a pass is re-run to narrow a key range
constexpr int NSUB = 256;
// re-run rounds of the user pass allowed inside one threshold selection
constexpr int MAX_REFINE = 4;
// smallest half-width of the window, in keys (2^12 ulps ~ 0.05 %)
constexpr int WMIN_BITS = 12;

// per-knapsack state of the threshold selection (device resident)
struct SelK {
    uint32_t ckey;        // centre key used by the last pass
    int32_t w;            // window half-width of the next pass: 2^w keys
    uint32_t wlo, whi;    // window [wlo, whi) used by the last pass
    uint32_t lo, hi;      // unresolved key range [lo, hi)
    unsigned long long above;  // fixed-point mass at or above hi
    int32_t state;        // 0 resolved, 1 needs a refine pass, 2 bucketed step (Sec. 5.2)
    uint32_t last_nz_key; // key of the last non-zero lambda_k (centre when lambda_k = 0)
    uint32_t for_key;     // key of the lambda_k the prediction below is for
    uint32_t pred_key;    // predicted key of the next lambda_k (centre of the next pass)
    uint32_t prev_key;    // key of the lambda_k before for_key
    float bdelta;         // bucket width Delta_k of a bucketed step (state 2)
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
    uint32_t ipath[KP_MAX_M];     // bit l set iff item j belongs to node l
    uint64_t items[KP_MAX_L];     // items of node l
    uint8_t cap[KP_MAX_L];        // C_l clamped to 255
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
    int32_t fixs;              // fixed-point shift of b sums: units of 2^-fixs
    float bscale;              // 2^fixs: the mass of an entry is round(b * bscale) <= 2^30
    int32_t fixo;              // fixed-point shift of the objective sums
    int32_t tile;              // dense: users per shared-memory tile
    int32_t stage;             // dense: 0 synchronous tile loads, 1 double-buffered bulk asynchronous copies
    int32_t creg;              // CSR: every item has exactly creg entries (0: not regular)
    int32_t vec;               // CSR regular rows aligned for vector loads (M in {8, 10, 16})
    int64_t uoff0;             // csr_user_off[0]
    double entries;            // b entries summed per knapsack (the count the unit 2^-fixs allows for)
    float maxb, maxp;          // largest b and p of the instance
    Tree tree;
};

// device scratch owned by a handle
struct Scratch {
    int32_t G;                        // persistent grid size of the user pass
    int32_t g_lo, gspan;              // blocks [g_lo, g_lo + gspan) can touch this instance
    int32_t cap_kb;                   // buffer entries per (k, block)
    unsigned long long *Rfix;         // [K]
    unsigned long long *objfix;       // [2] fixed-point dual and primal sums
    unsigned long long *reg3;         // [K][3] mass at/above, inside, below the window
    unsigned long long *subhist;      // [K][NSUB]
    uint2 *buf;                       // [K][gspan][cap_kb] (key, float bits of v2)
    uint32_t *bufcnt;                 // [K][gspan]
    uint32_t *ovf;                    // [K]
    SelK *sel;                        // [K]
    Counters *ctr;
    uint2 *shmask;                    // [N] CSR: .x entries whose knapsack another item of the user
                                      // also uses, .y up to PAIRS_MAX knapsacks exactly two items of
                                      // the user use (pair_first / pair_second / pair_count)
    const unsigned long long *rare;   // [nrare] CSR: (user << 5) | first entry, for the knapsacks
                                      // that three or more items of one user use
    int64_t nrare;
    int32_t rare_blk0, rare_grid;     // buffer blocks [rare_blk0, +rare_grid) of the rare-knapsack kernel
    const uint8_t *block;             // [K] device, knapsacks a block coordinate-descent step updates
                                      // (nullptr: all of them, Algorithm 4)
    const struct Scratch *peers;      // [npeers] device: the other shards of a user-sharded instance,
    int32_t npeers;                   // whose integer partials and buffers the lead's selection also reads
};

enum PassMode { MODE_STATE = 0, MODE_HIST = 1, MODE_REFINE = 2 };

// Many independent instances processed by one persistent launch: blocks take
// tiles from a shared counter; the tile list holds the most expensive
// instances first, each instance's tiles consecutive.
struct BatchDev {
    const Params *P;        // [count]
    Scratch *S;             // [count]
    const int64_t *koff;    // [count + 1] offsets of each instance's multipliers
    const int64_t *xoff;    // [count] offsets of each instance's x words
    const int32_t *kinst;   // [sum K] instance of every global knapsack index
    const uint8_t *solo;       // [count] 1: the instance runs its own passes (not in the tile list)
    const int32_t *tile_inst;  // [ntiles]
    const int64_t *tile_u0;    // [ntiles]
    unsigned long long *next;  // [MAX_REFINE + 1] tile counters, one per pass of a step
    int64_t ntiles;
    int32_t count;
};

// Knapsacks used by exactly two items of a user, listed in shmask.y: up to
// PAIRS_MAX (first entry, second entry) pairs of 5-bit entry indices, the count
// in the top two bits.  Further ones go to the rare-knapsack list.
constexpr int PAIRS_MAX = 3;
__host__ __device__ inline int pair_count(uint32_t y) { return (int)(y >> 30); }
__host__ __device__ inline int pair_first(uint32_t y, int t) { return (int)((y >> (10 * t)) & 31u); }
__host__ __device__ inline int pair_second(uint32_t y, int t) { return (int)((y >> (10 * t + 5)) & 31u); }

// Fixed-point unit 2^-s of the b masses: the mass round(b * 2^s) of one entry
// stays at most 2^30 (equal when max b is a power of two; one 32-bit
// conversion per entry) and every per-knapsack sum over `count` entries below
// 2^62.
inline int mass_shift(double count, float maxb) {
    const double lb = maxb > 0.f ? std::log2((double)maxb) : -200.0;
    const int s1 = (int)std::floor(62.0 - std::log2(count * (double)maxb + 1.0));
    const int s2 = 30 - (int)std::ceil(lb);
    int s = s1 < s2 ? s1 : s2;
    if (s > 40) s = 40;
    if (s < -120) s = -120;
    return s;
}

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
// bucketed Reduce (Sec. 5.2): the pass of round BUCKET_ROUND (re-run mode,
// every knapsack in state 2) bins every breakpoint by its bucket around
// lambda_k^t; the select interpolates inside the crossing bucket
constexpr int BUCKET_ROUND = 7;
cudaError_t launch_bucket_prep(const Params &P, const Scratch &S, const double *lambda, double delta,
                               cudaStream_t st);
cudaError_t launch_bucket_select(const Params &P, const Scratch &S, const double *lambda, double *lambda_next,
                                 cudaStream_t st);
cudaError_t launch_select(const Params &P, const Scratch &S, const double *lambda,
                          double *lambda_next, int round, cudaStream_t st);
cudaError_t launch_batch_pass(const BatchDev &B, int maxm, size_t smem, int grid, const double *lam,
                              int mode, int round, uint32_t *x_all, cudaStream_t st);
int batch_grid_size(int maxm, size_t smem);
size_t dense_smem_bytes(const Params &P, int mode);
int dense_tile_users(const Params &P);
cudaError_t launch_batch_finalize(const BatchDev &B, const double *lam, double *R, double *dual,
                                  double *primal, double alpha, double *lam_next, cudaStream_t st);
cudaError_t launch_batch_select(const BatchDev &B, int64_t totK, const double *lam,
                                double *lam_next, int round, cudaStream_t st);
cudaError_t launch_backward(const Params &P, const double *lambda, const uint32_t *x_bits,
                            const double *R, const double *upstream, double *grad_lambda,
                            float *grad_p, double *grad_B, cudaStream_t st);
cudaError_t launch_validate(const Params &P, uint32_t *flags, cudaStream_t st);
cudaError_t launch_wait_selftest(uint64_t limit_ns, int32_t *status, cudaStream_t st);
cudaError_t launch_shmask(const Params &P, uint2 *shmask, unsigned long long *rare, int64_t cap,
                          unsigned long long *count, cudaStream_t st);
// kp_api.cu
void set_last_error(const char *msg);

}  // namespace kp

// a problem handle (include/kp.h): parameters, scratch, and the allocations to free
struct kp_problem {
    kp::Params P;
    kp::Scratch S;
    int device;
    std::vector<void *> allocs;
    unsigned long long *ppbuf = nullptr;  // post-processing scratch, allocated at its first call
    size_t ppwords = 0;
};

namespace kp_impl {
// kp_api.cu: validation + parameters, and scratch for blocks [g_lo, g_lo + gspan)
kp_status prepare(const kp_desc *d, kp_problem *h);
// the checks and parameters of prepare, with the scan's five flag words given
// by the caller (device memory) and run on stream st; allocates nothing
kp_status fill_params(const kp_desc *d, kp::Params &P, uint32_t *flags, cudaStream_t st);
kp_status alloc_scratch(kp_problem *h, int G, int g_lo, int gspan, double budget, kp::Counters *ctr,
                        uint32_t *bufcnt = nullptr);
}  // namespace kp_impl
