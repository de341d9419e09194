// Batched COCG for the Sternheimer systems: shared declarations.
#pragma once
#include <algorithm>

#include "rpa_internal.cuh"

namespace rpa {

constexpr int kTile = 1024;  // grid points per block in the COCG kernels

// per-system scalar layout (doubles)
constexpr int kSysD = 16;
constexpr int kRho = 0, kAlpha = 2, kBeta = 4, kBnorm = 6, kTarget = 7, kRnorm = 8,
              kRnormTrue = 9;
// p^T V_nl p of the current direction (complex), from its projector coefficients (0 without
// projectors); the H-apply kernels sum p^T (H_loc - sigma) p and the alpha step adds it
constexpr int kNlDot = 10;
// per-system ints
constexpr int kSysI = 4;
constexpr int kStatus = 0, kIters = 1, kRestarts = 2,
              kIterBase = 3;  // kIters when the current COCG loop started
// statuses
constexpr int kActive = 0, kConverged = 1, kFinal = 2, kMaxit = 3, kBreakdown = 4, kIdle = 5;
constexpr int kNumStatus = 6;

template <typename T>
struct CocgView {
  Stencil<T> st;
  const T* vloc;
  NonlocalDev<T> nl;
  long long nd;
  int nsys, ns, tiles;
  const T* psi;          // ns x N_d
  const double* eps;     // ns
  const double* omega;   // per probe slot
  const T* u;            // per probe slot, N_d
  cpx<T>*x, *r, *p, *w;  // nsys x N_d
  cpx<T>* cdot;          // nsys x ngroup x 4
  double* part;          // nsys x tiles x 4
  double* sysd;          // nsys x kSysD
  int* sysi;             // nsys x kSysI
  const int* list;       // optional: compacted indices of the active systems (grid.y)
};

template <typename T>
cudaError_t proj_dots(const NonlocalDev<T>& nl, long long nd, int nsys, const cpx<T>* vec,
                      const int* sysi, int mask, cpx<T>* cd, cudaStream_t st);
template <typename T>
cudaError_t apply_h(const Stencil<T>& st, const T* vloc, const NonlocalDev<T>& nl, long long nd,
                    int count, const cpx<T>* x, const cpx<T>* sigma, cpx<T>* cd, cpx<T>* y,
                    cudaStream_t s);
// Double-float form of the mixed form's FP64 quantities (each value an unevaluated sum
// hi + lo of two floats, about 48 significant bits), so that the refinement residual runs
// on the FP32 units: the hi parts of the projector data are the FP32 copies.
struct DfAux {
  NonlocalDev<float> nl;    // hi parts: g_chi, p_chi, coef
  const float* g_chi_lo;    // lo parts of the group-major projector values
  const float* p_chi_lo;    // lo parts of the point-major projector values
  const float* coef_lo;     // lo parts of gamma dV
  const float2* vloc;       // (hi, lo) of V_loc, N_d
  const float2* psi;        // (hi, lo) of psi, ns x N_d
  const float2* u;          // (hi, lo) of u, per probe slot x N_d
};
// (hi, lo) pairs of a double array
cudaError_t convert_d2df(const double* a, float2* b, long long n, cudaStream_t s);
// mixed-form FP64 solution kept as double-float pairs (re.hi, re.lo, im.hi, im.lo):
// xh = xl (set) or xh += xl for the selected systems (as accumulate)
cudaError_t accumulate_df(long long nd, int nsys, const int* sysi, int mask, int round,
                          const cpx<float>* xl, float4* xh, int set, cudaStream_t s);
// dens_b = 4 sum_n psi_n (.) Re x_{b,n} from double-float x (FP64 sums)
cudaError_t density_df(long long nd, int ns, int nb, const double* psi, const float4* x,
                       const int* probe_active, double* dens, cudaStream_t s);
// projector coefficients gamma dV chi^T x of double-float x, in double-float sums, as FP64
cudaError_t proj_dots_df(const DfAux& aux, long long nd, int nsys, const float4* x,
                         const int* sysi, int mask, cpx<double>* cd, cudaStream_t s);

// With r_lo: the low-precision copy r_lo = r, x_lo = 0, and p_lo = r_lo (restart) -- or, with
// p_keep, the direction of the previous loop is kept for a continued recurrence: it is
// copied from p_keep into p_lo for systems whose last loop ran an odd number of iterations
// (their latest direction is in the other buffer of the pair), and p_lo = r_lo only for
// systems that did not iterate.
// For T = double, TL = float (the mixed form's refinement) x holds double-float pairs
// (float4 per complex value, see accumulate_df), r may be null (the FP64 residual is then
// not stored), and use_df needs aux: the whole residual then runs in double-float
// arithmetic; without use_df x is converted to FP64 as it is loaded.
template <typename T, typename TL>
cudaError_t cocg_resid(const CocgView<T>& cv, const cpx<T>* x, cpx<T>* r, cpx<T>* pdir, int mask,
                       cpx<TL>* r_lo, cpx<TL>* p_lo, cpx<TL>* x_lo, cudaStream_t s,
                       bool use_df = false, const cpx<TL>* p_keep = nullptr,
                       const DfAux* aux = nullptr);
// Per-system scalar step (kind: 0 init, 1 alpha, 2 beta/convergence, 3 true-residual
// recheck, 4 FP64 refinement check (restart), 5 mixed-form init, 6 FP64 refinement check
// continuing the recurrence: beta = rho(new true residual) / rho(last recursive step),
// 7 final FP64 check after the last refinement round: final, or not converged).  `tiles` partial sums per system are
// added; `stride` (default tiles) is the per-system stride of the partial-sum buffer.
// With list != null, nsys is the length of the list and the step runs for listed systems.
cudaError_t cocg_scalars(int nsys, int tiles, const double* part, double* sysd, int* sysi,
                         int kind, int mask, double tol, double inner_tol, int maxit,
                         int max_restart, cudaStream_t s, int stride = 0,
                         const int* list = nullptr);
// counts[status] over all systems; with list != null also writes the indices of the
// active systems (order unspecified) to list[0 .. counts[kActive])
cudaError_t count_status(int nsys, const int* sysi, int* counts, cudaStream_t s,
                         int* list = nullptr);
cudaError_t set_status(int nsys, int ns, const int* probe_active, int on, int* sysi,
                       cudaStream_t s);
// Loop control of a COCG loop captured as one graph (one thread).  ctl[0] counts the
// iterations run, ctl[1] the kernels launched: each adds its argument (0 for a pure check).
// Sets the while-node condition h to 1 while more than wnext systems are active
// (counts[kActive], as written by count_status) and ctl[0] <= limit, else 0.
cudaError_t loop_cond(const int* counts, unsigned long long* ctl, cudaGraphConditionalHandle h,
                      int wnext, int limit, int add_iters, int add_launches, cudaStream_t s);
cudaError_t remap_status(int nsys, int from, int to, int* sysi, cudaStream_t s);
template <typename TH, typename TL>
cudaError_t accumulate(long long nd, int nsys, const int* sysi, int mask, int round,
                       const cpx<TL>* xl, cpx<TH>* xh, int set, cudaStream_t s);
template <typename TX, typename TP>
cudaError_t density(long long nd, int ns, int nb, const TP* psi, const cpx<TX>* x,
                    const int* probe_active, double* dens, cudaStream_t s);

// dense.cu ----------------------------------------------------------------------------------
// Galerkin projection over the occupied space (Section 4):
//   G_b = -dV Psi diag(u_b) Psi^T  (N_s x N_s per probe slot b),
//   C_b[k][n] = G_b[k][n] / (eps_k - eps_n - i w_b),
//   x0_{b,n} = sum_k psi_k C_b[k][n].
template <typename T>
cudaError_t galerkin_guess(long long nd, int ns, int nb, const T* psi, const double* eps,
                           const double* omega, const T* u, const int* probe_active, double dV,
                           double* gpart, int nchunk, cpx<T>* cmat, cpx<T>* x0, cudaStream_t s);
// The same projection on the tensor cores (umma.cu, tcgen05 kind::tf32, 3-pass tf32 split):
// FP32 operands, FP32 results; err receives 1 if a bounded tensor-core wait expired
// (test_expire: make the first wait of every block expire, see umma.cu).
cudaError_t galerkin_guess_tc(long long nd, int ns, int nb, const float* psi, const double* eps,
                              const double* omega, const float* u, const int* probe_active,
                              double dV, double* gpart, int nchunk, cpx<float>* cmat,
                              cpx<float>* x0, int* err, cudaStream_t s, bool bf16 = false,
                              int test_expire = 0);
// Mode products along one axis of a batch of 3-D arrays: out[..a..] = sum_i Mt[i][a] in[..i..]
// (Mt is nin x nout, row-major).  dims_in = (nx, ny, nz) of the input; batch strides in_bs and
// out_bs.  Optional elementwise scale of the output (same layout as the output).
template <typename TI, typename TO, typename T>
cudaError_t mode_product(const TI* in, long long in_bs, TO* out, long long out_bs, const T* Mt,
                         int axis, const int* dims_in, int nout, int batch, const T* scale,
                         cudaStream_t s);
// Lanczos helpers (FP64): dots, combination, norm, normalisation
cudaError_t multi_dot(long long nd, int nb, const double* Q, long long ldq, int m0, int m1,
                      const double* v, const int* active, double* part, int nchunk,
                      double* dots, cudaStream_t s);
cudaError_t multi_axpy(long long nd, int nb, const double* Q, long long ldq, int m0, int m1,
                       const double* coef, int ldc, double* v, const int* active, cudaStream_t s);
cudaError_t convert_d2f(const double* a, float* b, long long n, cudaStream_t s);
cudaError_t convert_f2d(const float* a, double* b, long long n, cudaStream_t s);
cudaError_t jacobi_eig(double* a, double* v, double* lam, int n, cudaStream_t s);
cudaError_t jacobi_eig_batched(double* a, double* v, double* lam, const int* n, int count,
                               long long lda, long long ldl, cudaStream_t s);
// block Lanczos quadrature (lanczos_block.cu)
int block_max();
cudaError_t block_dot(long long nd, int nslot, int bmax, const int* bfirst, const int* bsize,
                      const double* Q, long long ldq, long long ldj, int j0, int nj,
                      const double* V, const int* active, double* part, int nchunk, double* D,
                      cudaStream_t s);
cudaError_t block_axpy(long long nd, int nslot, const int* bfirst, const int* bsize,
                       const double* Q, long long ldq, int nj, const double* D, int ldD,
                       double* V, const int* active, cudaStream_t s);
cudaError_t block_store_a(int nblk, const int* bstart, const int* bsz, const double* D, int ldD,
                          int nj, int k, int nl, double* Ab, const int* active, cudaStream_t s);
cudaError_t block_chol(int nblk, const int* bstart, const int* bsz, const double* G, int ldG,
                       int pass, int k, int nl, const double* Ab, double* Rk, double* Rinv,
                       double* Bb, int* active, int* bsteps, cudaStream_t s);
cudaError_t block_scale(long long nd, int nblk, const int* bstart, const int* bsz,
                        const double* Rinv, const double* V, double* out, long long ldo,
                        const int* active, cudaStream_t s);
cudaError_t block_quadrature(int nblk, const int* bstart, const int* bsz, const int* bsteps,
                             int steps_all, int nl, const double* Ab, const double* Bb, double* T,
                             double* W, double* lam, long long ldT, long long ldl, int* mdim,
                             int fkind, double* dout, cudaStream_t s);

}  // namespace rpa
