// Per-probe FP64 kernels: declarations.
#pragma once
#include "rpa_internal.cuh"

namespace rpa {

cudaError_t tridiag_f11(int count, int k, const double* alpha, int lda, const double* beta,
                        int ldb, const int* kper, int fkind, double* d, cudaStream_t s);
cudaError_t gl_nodes(int nw, double* omega, double* weight, cudaStream_t s);
cudaError_t interp_matrix(int n, int m, int bc, int kind, const long long* nodes, double* Wt,
                          cudaStream_t s);
cudaError_t ec_reduce(long long nd, int nw, const double* dfine, const double* weight,
                      double* part, int nblk, double* ec, cudaStream_t s);
cudaError_t nu_scale(const double* l0, const double* l1, const double* l2, int nx, int ny, int nz,
                     double lmax, double* s64, float* s32, cudaStream_t s);
cudaError_t lanczos_alpha(int nb, int k, int nl, const double* dots, const int* active,
                          double* alpha, const double* beta, double* coef, cudaStream_t s);
cudaError_t lanczos_beta(int nb, int k, int nl, const double* vnorm2, int* active, double* alpha,
                         double* beta, int* steps, double* lstate, double lrtol, int fkind,
                         int* flags, cudaStream_t s);
cudaError_t lanczos_next(long long nd, int nb, int k, int nl, const int* active,
                         const double* lstate, const double* beta, const double* v, double* Q,
                         long long ldq, cudaStream_t s);
cudaError_t lanczos_start(long long nd, int nb, const long long* probe, double* Q, long long ldq,
                          cudaStream_t s);

}  // namespace rpa
