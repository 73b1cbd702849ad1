/*
 * kp.h -- C ABI of the GB300 dual-decomposition knapsack library
 * (method of Zhang, Qi, Hua, Yang, "Solving Billion-Scale Knapsack Problems",
 * WWW 2020, arXiv 2002.00352).
 *
 * Problem (Sec. 2, Eq. (1)-(4)): N users ("groups"), M items per user, K
 * global knapsacks, L local count constraints shared by all users:
 *
 *     max  sum_ij p_ij x_ij
 *     s.t. sum_ij b_ijk x_ij <= B_k            for every knapsack k
 *          sum_{j in S_l} x_ij <= C_l          for every user i and set l
 *          x_ij in {0, 1}
 *
 * with p, b >= 0 and B, C > 0.  The local sets must be hierarchical
 * (Sec. 2.1, Definition 1: any two are disjoint or nested); the per-user
 * subproblem at fixed multipliers (Eq. (11)-(13)) is then solved exactly by
 * the greedy of Algorithm 1.
 *
 * Conventions shared by every call:
 *   - "device" pointers are CUDA global memory of the current device; the
 *     caller owns all of them.  kp_create borrows the instance arrays: they
 *     must stay allocated and unchanged (except B, see below) until
 *     kp_destroy.  The handle owns only its scratch memory.
 *   - Every compute call is asynchronous on the given stream (a
 *     cudaStream_t passed as void*; NULL = legacy default stream).  Outputs
 *     are valid after the stream has been synchronised.
 *   - Multipliers lambda are FP64 [K] device arrays with lambda_k >= 0
 *     (Eq. (10)).  Kernels round lambda to FP32 once per call; reduced costs
 *     and breakpoints are computed in FP32, all sums over users in FP64 or
 *     exact 64-bit fixed point.
 *   - Consumption b is summed in units of 2^-s, each entry rounded once to
 *     the nearest unit, with s = min(40, 30 - ceil(log2 max b),
 *     floor(62 - log2(entries * max b + 1))) (at least -120) chosen at
 *     kp_create: the largest b keeps 30 bits unless it is below 2^-10, and
 *     with s = 40 entries up to 2^-41 count as 0.
 *   - Calls on one handle must be ordered on one stream (they share the
 *     handle's scratch).
 *   - Return value: KP_OK, or an error code with nothing written to any
 *     output; kp_last_error() then describes the error (thread-local).
 *     Errors detected by a kernel (a bounded wait that ran out, a selection
 *     that did not converge) are reported by kp_device_status().
 *   - No C++ exception crosses this interface.
 */
#ifndef KP_H
#define KP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    KP_OK = 0,
    KP_EINVAL = 1,   /* invalid argument or instance (sizes, tree, caps) */
    KP_ENOMEM = 2,   /* device allocation failed */
    KP_ECUDA = 3,    /* a CUDA runtime call failed */
    KP_ETIMEOUT = 4, /* a kernel's bounded wait ran out (device status) */
    KP_ESTATE = 5,   /* inconsistent state, e.g. threshold search did not converge */
    KP_EDATA = 6     /* instance data violate Sec. 2 (negative or non-finite p, b;
                        B <= 0; malformed CSR) */
} kp_status;

enum { KP_B_DENSE = 0, KP_B_CSR = 1 };

/* limits of this implementation */
enum { KP_MAX_M = 64, KP_MAX_L = 16, KP_MAX_K = 2048 };

typedef struct kp_problem kp_problem;

/* Instance description (Sec. 2, Eq. (1)-(4)).
 *
 *   N, M, K      users, items per user (1..KP_MAX_M), knapsacks (1..KP_MAX_K)
 *   p            device float32 [N*M], p_ij at i*M+j, >= 0
 *   b_layout     KP_B_DENSE or KP_B_CSR
 *   b_dense      device float32 [N*M*K], b_ijk at (i*M+j)*K+k, >= 0
 *   csr_user_off device int64 [N+1]: entries of user i are
 *                [csr_user_off[i], csr_user_off[i+1]) of csr_val / csr_k
 *   csr_item_nnz device uint8 [N*M]: the entries of user i are grouped by
 *                item in item order; item j owns csr_item_nnz[i*M+j] of them
 *   csr_val      device float32 [nnz] b_ijk of the entry, >= 0
 *   csr_k        device int16 [nnz] k of the entry, 0 <= k < K, strictly
 *                increasing within an item
 *   B            device float64 [K], B_k > 0.  Read at every call, so the
 *                caller may change the budgets between calls (e.g. an outer
 *                gradient loop on B).
 *   L            number of local constraints (0..KP_MAX_L)
 *   S            host uint64 [L]: bit j of S[l] set iff item j is in S_l
 *   C            host int32 [L]: caps C_l >= 1 (Eq. (3))
 *   S and C are copied at kp_create.
 */
typedef struct {
    int64_t N;
    int32_t M;
    int32_t K;
    const float *p;
    int32_t b_layout;
    const float *b_dense;
    const int64_t *csr_user_off;
    const uint8_t *csr_item_nnz;
    const float *csr_val;
    const int16_t *csr_k;
    const double *B;
    int32_t L;
    const uint64_t *S;
    const int32_t *C;
} kp_desc;

/* Validates the description (sizes, hierarchical sets per Sec. 2.1, caps),
 * scans the instance once on the device (p, b finite and >= 0; CSR offsets
 * consistent with item counts, k in range and increasing per item; B > 0),
 * allocates the scratch and returns a handle in *out.  Synchronous.
 * KP_EINVAL / KP_EDATA / KP_ENOMEM / KP_ECUDA on failure (*out untouched). */
kp_status kp_create(const kp_desc *desc, kp_problem **out);

/* Frees the handle's scratch.  Synchronises the device.  NULL is a no-op. */
kp_status kp_destroy(kp_problem *h);

/* Per-user decisions at lambda: Algorithm 1 for every user (Sec. 4.2).
 * x_bits: device uint32 [N*W], W = ceil(M/32); bit (j%32) of word
 * i*W + j/32 is x_ij. */
kp_status kp_solve_users(kp_problem *h, const double *lambda, uint32_t *x_bits, void *stream);

/* Map + Reduce of Algorithm 2 at lambda: R_k = sum_i sum_j b_ijk x_ij
 * (device float64 [K]), dual_sum = sum_ij p~_ij x_ij, primal_sum =
 * sum_ij p_ij x_ij and g = dual_sum + sum_k lambda_k B_k (the dual
 * objective, Eq. (5)) (device float64 scalars).  x_bits as in
 * kp_solve_users; every output pointer may be NULL. */
kp_status kp_reduce_consumption(kp_problem *h, const double *lambda, double *R,
                                double *dual_sum, double *primal_sum, double *g,
                                uint32_t *x_bits, void *stream);

/* Dual objective (Eq. (5)): g(lambda) = sum_i max_x sum_j p~_ij x_ij + sum_k lambda_k B_k,
 * written to the device float64 scalar g. */
kp_status kp_dual_value(kp_problem *h, const double *lambda, double *g, void *stream);

/* One dual-descent iteration (Eq. (14), Algorithm 2):
 * lambda_next_k = max(lambda_k + alpha (R_k - B_k), 0).  lambda_next may
 * alias lambda.  R (device [K]) may be NULL. */
kp_status kp_dd_step(kp_problem *h, const double *lambda, double alpha, double *lambda_next,
                     double *R, void *stream);

/* Map of Algorithm 4 (the step functions that Algorithm 3's candidates
 * describe) at lambda: every user's breakpoints of its k-consumption in
 * lambda_k (others fixed) are aggregated into the handle's per-knapsack
 * masses around a predicted threshold (Sec. 5.2 centres its buckets at
 * lambda_k), the ones close to it buffered.  The state at lambda is reduced
 * in the same pass into the optional outputs (as in kp_reduce_consumption);
 * for CSR rows with the same number of entries per item, R is the mass of
 * the breakpoints above lambda_k, which equals the consumption up to users
 * whose reduced costs tie within FP32 rounding.  Must be followed by
 * kp_threshold_select with the same lambda.  KP_EINVAL when the per-knapsack
 * state does not fit in shared memory (K near KP_MAX_K with more than 10
 * items per user). */
kp_status kp_scd_breakpoints(kp_problem *h, const double *lambda, double *R, double *dual_sum,
                             double *primal_sum, uint32_t *x_bits, void *stream);

/* Reduce of Algorithm 4 for every k:
 *   lambda_next_k = min { v in {0} U {breakpoints} : sum_{v1 > v} v2 <= B_k }
 * found exactly among the FP32 breakpoints (window masses, then a buffered
 * exact selection; when the crossing lies outside the buffered window the
 * user pass is re-run to narrow it, up to a fixed number of rounds, all on
 * the device).  lambda must be the one given to kp_scd_breakpoints.
 * lambda_next must not alias lambda. */
kp_status kp_threshold_select(kp_problem *h, const double *lambda, double *lambda_next, void *stream);

/* One full iteration of Algorithm 4: kp_scd_breakpoints + kp_threshold_select. */
kp_status kp_scd_step(kp_problem *h, const double *lambda, double *lambda_next, double *R,
                      double *dual_sum, double *primal_sum, void *stream);

/* One block coordinate-descent iteration (Sec. 4.3.2, the variants of
 * Algorithm 4 that update one multiplier, cyclic CD, or a block of them, block
 * CD): for every k with block[k] != 0 (block: device uint8 [K]) the Reduce of
 * Algorithm 4 at lambda,
 *   lambda_next_k = min { v in {0} U {breakpoints} : sum_{v1 > v} v2 <= B_k },
 * and lambda_next_k = lambda_k for the others.  Only the breakpoints of the
 * block's knapsacks are computed.  With every block[k] = 1 this is
 * kp_scd_step; with one k it is a step of cyclic CD.  dual_sum and
 * primal_sum (nullable) as in kp_scd_breakpoints; lambda_next must not alias
 * lambda. */
kp_status kp_bcd_step(kp_problem *h, const double *lambda, const uint8_t *block, double *lambda_next,
                      double *dual_sum, double *primal_sum, void *stream);

/* One iteration of Algorithm 4 whose Reduce is the bucketing with
 * interpolation of Sec. 5.2 (an approximation of the exact Reduce above).
 * Every breakpoint v of knapsack k goes to the bucket
 *   id(v) = 0 if |v - lambda_k| < Delta_k,
 *           else sign(v - lambda_k) (1 + floor(log2(|v - lambda_k| / Delta_k)))
 * (narrowest at lambda_k = lambda_k^t, doubling away from it; clamped to
 * [-127, 127]; computed in FP32 from the FP32 breakpoint, lambda_k rounded
 * to FP32 and Delta_k), with Delta_k = delta * lambda_k, or delta where
 * lambda_k = 0.  Walking down from the highest bucket, the first bucket
 * whose mass takes the cumulative mass above B_k holds lambda_next_k; inside
 * it the mass is taken as uniform over the bucket's range
 *   id 0: [lambda_k - Delta_k, lambda_k + Delta_k),
 *   id > 0: [lambda_k + Delta_k 2^(id-1), lambda_k + Delta_k 2^id),
 *   id < 0: [lambda_k - Delta_k 2^|id|, lambda_k - Delta_k 2^(|id|-1)),
 * and lambda_next_k is the point where the cumulative mass reaches B_k
 * (clamped to the bucket and to >= 0); lambda_next_k = 0 when the whole
 * emitted mass is within B_k.  Bucket masses are exact fixed-point sums.
 * One user pass per call, no re-run passes.  lambda, lambda_next: device
 * FP64 [K], must not alias.  KP_EINVAL for delta outside (0, 1e30].  Leaves
 * the exact Reduce's threshold prediction untouched. */
kp_status kp_scd_step_bucketed(kp_problem *h, const double *lambda, double delta, double *lambda_next,
                               void *stream);

/* Gradient of the dual g(lambda, p, B) of Eq. (5) by Danskin's theorem at the
 * maximiser x* (from kp_solve_users / kp_reduce_consumption at the same
 * lambda), each scaled by the device float64 scalar *upstream:
 *   grad_lambda_k = upstream (B_k - R_k)       (R from the same lambda)
 *   grad_p_ij     = upstream x*_ij             (device float32 [N*M])
 *   grad_B_k      = upstream lambda_k
 * Any of the three outputs may be NULL.  (The paper gives no gradient; this
 * is the derivative of its dual function, Eq. (5).) */
kp_status kp_dual_backward(kp_problem *h, const double *lambda, const uint32_t *x_bits,
                           const double *R, const double *upstream, double *grad_lambda,
                           float *grad_p, double *grad_B, void *stream);

/* ------------------------------------------------------------------------
 * Batches: many independent instances (each its own Eq. (1)-(4) problem, with
 * its own N, M, K, sets and budgets) solved together.  Every pass over the
 * users of all instances is one persistent kernel launch over a work list of
 * (instance, tile of users); the selection runs one block per (instance,
 * knapsack).  The paper solves one instance at a time; batching is this
 * library's way to keep the GPU busy with many small ones.
 *   - Multipliers of the batch: one float64 device array, instance i's K_i
 *     values at offset koff[i] (kp_batch_layout); same for R.
 *   - x_bits: instance i's N_i * ceil(M_i/32) words follow instance i-1's.
 *   - dual_sum / primal_sum: one float64 per instance.
 *   - Only dense instances (KP_B_DENSE) can be batched (KP_EINVAL otherwise).
 * Instance data are borrowed as in kp_create; validation as in kp_create.
 * ------------------------------------------------------------------------ */
typedef struct kp_batch kp_batch;

kp_status kp_batch_create(const kp_desc *descs, int32_t count, kp_batch **out);
kp_status kp_batch_destroy(kp_batch *b);
/* koff: host int64 [count + 1], offsets of each instance's multipliers. */
kp_status kp_batch_layout(kp_batch *b, int64_t *koff);
/* kp_reduce_consumption for every instance (Algorithm 2 Map + Reduce). */
kp_status kp_batch_reduce_consumption(kp_batch *b, const double *lambda, double *R,
                                      double *dual_sum, double *primal_sum, uint32_t *x_bits,
                                      void *stream);
/* kp_dd_step (Eq. (14)) for every instance with the same alpha. */
kp_status kp_batch_dd_step(kp_batch *b, const double *lambda, double alpha, double *lambda_next,
                           void *stream);
/* kp_scd_step (Algorithms 3-4) for every instance; lambda_next must not alias lambda. */
kp_status kp_batch_scd_step(kp_batch *b, const double *lambda, double *lambda_next, void *stream);
/* As kp_device_status, over every instance of the batch. */
kp_status kp_batch_device_status(kp_batch *b, void *stream);

/* ------------------------------------------------------------------------
 * User-sharded instances: one instance whose users are split over several
 * handles (shards; on several GPUs, one per device), solved as one.  Users are
 * independent given lambda (Sec. 4.1, the Map of Algorithms 2 and 4), so each
 * shard runs the user passes of its own users and the Reduce combines the
 * shards' exact integer partials (fixed-point consumption and objective sums,
 * window masses, sub-histograms) and their buffered breakpoints: the result is
 * that of one handle over all the users, bit for bit.
 *   - Each shard is created with kp_create over its range of users (p, b and
 *     the CSR rows of those users; the same K, M, local sets and budgets B).
 *   - kp_shard_group_create sets one fixed-point unit for all shards (the one
 *     a single handle would choose for the union) and keeps the handles; they
 *     must outlive the group and be used through it only.  All shards must be
 *     on the current device (the lead's kernels read the others' scratch).
 *   - kp_shard_group_scd_step is kp_scd_step over the union; the selection
 *     state lives in shard 0 (the lead) and is copied to the others.
 * ------------------------------------------------------------------------ */
typedef struct kp_shard_group kp_shard_group;

kp_status kp_shard_group_create(kp_problem *const *shards, int32_t n, kp_shard_group **out);
kp_status kp_shard_group_destroy(kp_shard_group *g);
kp_status kp_shard_group_scd_step(kp_shard_group *g, const double *lambda, double *lambda_next, double *R,
                                  double *dual_sum, double *primal_sum, void *stream);

/* Allocation-free form of kp_reduce_consumption, for callers that cannot
 * allocate device memory: a process whose device memory belongs to its own
 * pool (an outside cudaMalloc would fail or fragment it), or code on a
 * latency-critical path that must not take the driver's allocation locks.
 * There is no counterpart in the paper; it computes exactly what
 * kp_reduce_consumption computes (same kernels), with no handle: the
 * instance is described by desc at every call and nothing is allocated.
 *   - Scratch: one file-scope __device__ array of (KP_MAX_K + 5) 64-bit
 *     words (about 16 KB) per device, kept by every device that loads the
 *     library until the process exits.  K > KP_MAX_K is rejected
 *     (KP_EINVAL).
 *   - The first call on a device looks up the array's device address (once
 *     per device); make that first call before any stream capture.
 *   - Each call clears the array, scans the instance as kp_create does
 *     (KP_EDATA on violations) and waits on `stream` for that scan's result,
 *     then enqueues the pass and returns; the outputs are valid after the
 *     stream has been synchronised.
 *   - Every call shares the array: calls that overlap on the GPU (other
 *     streams, other host threads) race and must be serialised by the caller.
 * Arguments and outputs as in kp_create and kp_reduce_consumption. */
kp_status kp_reduce_consumption_noalloc(const kp_desc *desc, const double *lambda, double *R,
                                        double *dual_sum, double *primal_sum, double *g,
                                        uint32_t *x_bits, void *stream);

/* Autotuner: times the breakpoint pass of a dense instance on its first
 * min(N, 2^18) users at several tile sizes (users staged per shared-memory
 * tile: the default, 8, 16, 32, 64, 128, 256 where they fit) in both staging
 * modes (kp_set_tile) and keeps the fastest pair for every later call on the
 * handle; *chosen (may be NULL) receives the tile size.  KP_ETIMEOUT if a
 * timed pass reported one.  A CSR instance has no run-time tile size (*chosen = 0).  Synchronous;
 * allocates K doubles for the duration of the call.  (Not in the paper.) */
kp_status kp_autotune(kp_problem *h, int32_t *chosen, void *stream);

/* Dense instances: the users per shared-memory tile (1 .. the default, which
 * fills a 64 KB tile of b and at most 96 KB of everything staged per user;
 * 0 = the default) and the staging mode of the user passes:
 * 0 = each tile loaded by the block's threads, then computed (two blocks per
 * SM overlap one's loads with the other's work); 1 = two buffers of half a
 * tile each, the next tile's p and b brought in by 1-D bulk asynchronous
 * copies (cp.async.bulk, completion on an mbarrier, waits bounded at 2 s:
 * KP_ETIMEOUT in kp_device_status) while the current one is computed; used
 * when p and b are 16-byte aligned and half a tile holds at least 4 users,
 * otherwise mode 0.  Results do not depend on either choice.  KP_EINVAL for
 * a CSR instance or values out of range.  (Not in the paper.) */
kp_status kp_set_tile(kp_problem *h, int32_t users, int32_t staging);

/* Exercises the bounded wait of staging mode 1 without a fault: one block
 * waits on an mbarrier that nothing arrives on, gives up after limit_ns
 * nanoseconds (1e3 .. 1e9) and reports KP_ETIMEOUT through its status word,
 * leaving the context usable.  Returns KP_ETIMEOUT (the expected outcome),
 * KP_OK if the wait completed (it cannot), KP_EINVAL for a limit out of
 * range.  Synchronous; allocates 4 bytes for the call. */
kp_status kp_wait_selftest(int64_t limit_ns, void *stream);

/* Synchronises the stream and returns the device-side status accumulated by
 * the handle's kernels since the last call (KP_OK, KP_ETIMEOUT or
 * KP_ESTATE), then clears it.  KP_ETIMEOUT: a dense user pass waited more
 * than 2 s for the bulk asynchronous copy of a tile of users into shared
 * memory (the block then stops, after waiting for its copies in flight; the
 * pass's results are incomplete). */
kp_status kp_device_status(kp_problem *h, void *stream);

/* Counters of the last kp_threshold_select on this handle (device values,
 * copied synchronously): out[0] = user passes run for the selection
 * (1 = resolved from the buffered window), out[1] = knapsacks resolved
 * from the histogram alone (lambda = 0), out[2] = buffer overflows. */
kp_status kp_select_stats(kp_problem *h, int64_t out[3], void *stream);

/* Pre-solving by sampling (Sec. 5.3): iters iterations of Algorithm 4 from
 * lambda = 0 on the users users[0..n) (device int64 [n], each in 0..N-1,
 * drawn by the caller, e.g. uniformly without replacement) with every budget
 * scaled by n / N; the result, a starting point for the whole instance, is
 * written to lambda0 (device float64 [K]).  The sample's rows are gathered
 * into buffers of its own and a handle is created over them for the call
 * (allocates; synchronous).  KP_EINVAL for a bad argument or an index
 * outside 0..N-1. */
kp_status kp_presolve(kp_problem *h, const int64_t *users, int64_t n, int32_t iters, double *lambda0,
                      void *stream);

/* Post-processing for feasibility (Sec. 5.4).  Users are taken in
 * non-decreasing order of their cost-adjusted group profit
 *     q_i = sum_{j : x_ij = 1} (p_ij - sum_k lambda_k b_ijk)
 * (q_i in FP64, items in ascending j and each item's knapsacks in ascending
 * k, every product and sum rounded to nearest; equal q_i: lower i first), and
 * every decision of a user is reset, in that order, until no knapsack exceeds
 * its budget (the users reset form the shortest such prefix; none if x is
 * already feasible).
 *   lambda   device float64 [K]: the multipliers that define q_i
 *   x_bits   device uint32 [N*W] as in kp_solve_users, any decisions; the
 *            reset users' words are zeroed in place, the others untouched
 *   reset    device int64 scalar: number of users reset (nullable)
 *   R_after  device float64 [K]: consumption of the returned x, summed in
 *            the fixed point of kp_reduce_consumption (nullable)
 * Budgets are compared in that fixed point (units of 2^-s with every entry's
 * b at most 2^30 units).  Asynchronous on the stream, except the first call
 * on a handle, which allocates 24 N + O(K) bytes of device memory (keys and
 * two lists of users) that the handle keeps until kp_destroy.  An
 * inconsistent selection (not expected) is reported as KP_ESTATE by
 * kp_device_status. */
kp_status kp_postprocess(kp_problem *h, const double *lambda, uint32_t *x_bits, int64_t *reset,
                         double *R_after, void *stream);

/* Launch layout of a handle (host values, no device work): out[0] = blocks of
 * the user pass, out[1] = users whose knapsacks shared by three or more of
 * their items are swept by a separate kernel (CSR; each breakpoint pass then
 * launches one more kernel), out[2] = blocks of that kernel (0 if none),
 * out[3] = breakpoint-buffer entries per (knapsack, block). */
kp_status kp_info(kp_problem *h, int64_t out[4]);

/* Limits of this implementation (host values, no device work): out[0] =
 * KP_MAX_M, out[1] = KP_MAX_L, out[2] = KP_MAX_K.  KP_EINVAL if out is NULL.
 * (Not in the paper.) */
kp_status kp_limits(int32_t out[3]);

/* Thread-local description of the last error on this thread. */
const char *kp_last_error(void);

/* Library version, major*10000 + minor*100 + patch. */
int kp_version(void);

#ifdef __cplusplus
}
#endif
#endif /* KP_H */
