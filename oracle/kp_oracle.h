/*
 * kp_oracle.h -- declarations of the FP64 CPU oracle (test infrastructure
 * only; see kp_oracle.c for what each routine follows in the paper).
 */
#ifndef KP_ORACLE_H
#define KP_ORACLE_H
#include <stdint.h>

void kpo_reduced_costs(int M, int K, const double *p, const double *b,
                       const double *lam, double *pt);
void kpo_topo_order(int L, const uint64_t *S, int *topo);
int kpo_is_hierarchical(int L, const uint64_t *S);
void kpo_greedy(int M, int L, const uint64_t *S, const int *C, const int *topo,
                const double *pt, int *x);
double kpo_brute_force(int M, int L, const uint64_t *S, const int *C,
                       const double *pt, int *x);
void kpo_user_pass(int64_t N, int M, int K, const double *p, const double *b,
                   int L, const uint64_t *S, const int *C, const double *lam,
                   int *x, double *R, double *dual, double *primal);
void kpo_dd_update(int K, const double *lam, const double *R, const double *B,
                   double alpha, double *lam_next);
double kpo_dual_value(int64_t N, int M, int K, const double *p,
                      const double *b, int L, const uint64_t *S, const int *C,
                      const double *lam, const double *B);
void kpo_scd_map_user(int M, int K, const double *pi, const double *bi, int L,
                      const uint64_t *S, const int *C, const int *topo,
                      const double *lam, int64_t *n, int32_t *ek, double *ev1,
                      double *ev2);
double kpo_scd_reduce(int64_t n, const double *v1, const double *v2, double Bk);
int64_t kpo_scd_step(int64_t N, int M, int K, const double *p, const double *b,
                     int L, const uint64_t *S, const int *C, const double *lam,
                     const double *B, double *lam_next, int64_t *nemit,
                     double *mass);
int64_t kpo_scd_map_all(int64_t N, int M, int K, const double *p, const double *b,
                        int L, const uint64_t *S, const int *C, const double *lam,
                        int64_t cap_out, int64_t *eu, int32_t *ek, double *ev1,
                        double *ev2);
int64_t kpo_postprocess(int64_t N, int M, int K, const double *p,
                        const double *b, const double *lam, const double *B,
                        int *x);
void kpo_alg5_map_user(int K, const double *pi, const double *bi, int Q,
                       const double *lam, int64_t *n, int32_t *ek,
                       double *ev1, double *ev2);
int64_t kpo_alg5_step(int64_t N, int K, const double *p, const double *bd,
                      int Q, const double *lam, const double *B,
                      double *lam_next);
int kpo_num_threads(void);

#endif
