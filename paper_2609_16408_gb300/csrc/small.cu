// Per-probe FP64 kernels: the tridiagonal eigen-problem behind [f(T)]_{11} (Eq. 7,
// Algorithm 1), the frequency rule (Eq. 9), interpolation operators (Section 3.2), the
// E_c reduction, and the spectral scale of nu^{1/2}.
#include <cuda_runtime.h>
#include <float.h>

#include "cocg.cuh"
#include "small.cuh"

namespace rpa {

// Eigenvalues (returned in a) and first components of the normalised eigenvectors (in z) of
// the symmetric tridiagonal matrix with diagonal a[0..k-1] and off-diagonal e[0..k-2]
// (e is destroyed).  Implicit symmetric QR steps with the Wilkinson shift of the trailing
// 2x2 block, chasing the bulge with Givens rotations; the first row of the accumulated
// rotation product is carried along.  Returns false if an eigenvalue needs > 60 steps.
__device__ bool tridiag_qr(int k, double* a, double* e, double* z) {
  for (int i = 0; i < k; ++i) z[i] = (i == 0) ? 1.0 : 0.0;
  int m = k - 1, steps = 0;
  while (m > 0) {
    if (fabs(e[m - 1]) <= DBL_EPSILON * (fabs(a[m - 1]) + fabs(a[m]))) {
      e[m - 1] = 0.0;
      --m;
      steps = 0;
      continue;
    }
    if (++steps > 60) return false;
    int l = m - 1;
    while (l > 0 && fabs(e[l - 1]) > DBL_EPSILON * (fabs(a[l - 1]) + fabs(a[l]))) --l;
    // Wilkinson shift: eigenvalue of the trailing 2x2 block nearer to a[m]
    const double dlt = 0.5 * (a[m - 1] - a[m]);
    const double em = e[m - 1];
    const double sg = (dlt >= 0.0) ? 1.0 : -1.0;
    const double mu = a[m] - em * em / (dlt + sg * hypot(dlt, em));
    double x = a[l] - mu, y = e[l];
    for (int i = l; i < m; ++i) {
      const double r = hypot(x, y);
      double c = 1.0, s = 0.0;
      if (r != 0.0) {
        c = x / r;
        s = y / r;
      }
      if (i > l) e[i - 1] = r;
      const double ai = a[i], ai1 = a[i + 1], ei = e[i];
      a[i] = c * c * ai + 2.0 * c * s * ei + s * s * ai1;
      a[i + 1] = s * s * ai - 2.0 * c * s * ei + c * c * ai1;
      e[i] = c * s * (ai1 - ai) + (c * c - s * s) * ei;
      if (i + 1 < m) {
        x = e[i];
        y = s * e[i + 1];
        e[i + 1] = c * e[i + 1];
      }
      const double z0 = z[i], z1 = z[i + 1];
      z[i] = c * z0 + s * z1;
      z[i + 1] = -s * z0 + c * z1;
    }
  }
  return true;
}

__device__ __forceinline__ double fapply(double x, int fkind) {
  if (fkind == RPA_F_X) return x;
  if (fkind == RPA_F_X2) return x * x;
  return log1p(-x) + x;
}

// d[i] = [f(T_i)]_{11}, T_i of order kper[i] (or k), one thread per tridiagonal.
__global__ void k_tridiag_f11(int count, int k, const double* __restrict__ alpha, int lda,
                              const double* __restrict__ beta, int ldb,
                              const int* __restrict__ kper, int fkind, double* __restrict__ d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  int kk = kper ? kper[i] : k;
  if (kk <= 0) return;
  double a[kMaxLanczos], e[kMaxLanczos], z[kMaxLanczos];
  for (int j = 0; j < kk; ++j) {
    a[j] = alpha[(long long)i * lda + j];
    e[j] = (j + 1 < kk) ? beta[(long long)i * ldb + j] : 0.0;
  }
  double out;
  if (!tridiag_qr(kk, a, e, z)) {
    out = __longlong_as_double(0x7ff8000000000000ULL);
  } else {
    out = 0.0;
    for (int j = 0; j < kk; ++j) out += z[j] * z[j] * fapply(a[j], fkind);
  }
  d[i] = out;
}

cudaError_t tridiag_f11(int count, int k, const double* alpha, int lda, const double* beta,
                        int ldb, const int* kper, int fkind, double* d, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_tridiag_f11<<<(count + 63) / 64, 64, 0, s>>>(count, k, alpha, lda, beta, ldb, kper, fkind, d);
  note_launch();
  return cudaGetLastError();
}

// Gauss-Legendre nodes/weights by the Golub-Welsch construction: the nodes are the
// eigenvalues of the Jacobi matrix of the Legendre recurrence (zero diagonal, off-diagonal
// j / sqrt(4 j^2 - 1)), the weights 2 z_1^2.  Mapped to [0, inf) by w = (1 + x)/(1 - x) with
// weight 2 w_GL / (1 - x)^2; nodes ordered by decreasing x.
__global__ void k_gl_nodes(int nw, double* omega, double* weight) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double a[64], e[64], z[64];
  for (int j = 0; j < nw; ++j) {
    a[j] = 0.0;
    const double jj = j + 1;
    e[j] = (j + 1 < nw) ? jj / sqrt(4.0 * jj * jj - 1.0) : 0.0;
  }
  if (!tridiag_qr(nw, a, e, z)) {
    for (int j = 0; j < nw; ++j) omega[j] = weight[j] = __longlong_as_double(0x7ff8000000000000ULL);
    return;
  }
  for (int i = 0; i < nw; ++i) {  // selection sort, decreasing node
    int best = i;
    for (int j = i + 1; j < nw; ++j)
      if (a[j] > a[best]) best = j;
    const double ta = a[i], tz = z[i];
    a[i] = a[best];
    z[i] = z[best];
    a[best] = ta;
    z[best] = tz;
  }
  for (int j = 0; j < nw; ++j) {
    const double x = a[j], w = 2.0 * z[j] * z[j];
    omega[j] = (1.0 + x) / (1.0 - x);
    weight[j] = 2.0 * w / ((1.0 - x) * (1.0 - x));
  }
}

cudaError_t gl_nodes(int nw, double* omega, double* weight, cudaStream_t s) {
  k_gl_nodes<<<1, 32, 0, s>>>(nw, omega, weight);
  note_launch();
  return cudaGetLastError();
}

// Transposed 1-D interpolation matrix Wt (m coarse x n fine): fine_i = sum_j Wt[j][i] c_j.
// kind: RPA_INTERP_NONE (identity, g = 1), TRILINEAR (2-point Lagrange), TRICUBIC (4-point
// Lagrange), FOURIER (zero-padded trigonometric interpolation, periodic, n = m g).
__global__ void k_interp_matrix(int n, int m, int bc, int kind, const long long* __restrict__ nodes,
                                double* __restrict__ Wt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int j = 0; j < m; ++j) Wt[(long long)j * n + i] = 0.0;
  if (m == 1) {
    Wt[i] = 1.0;
    return;
  }
  if (kind == RPA_INTERP_NONE) {
    Wt[(long long)i * n + i] = 1.0;
    return;
  }
  if (kind == RPA_INTERP_FOURIER) {
    const int g = n / m;
    const int K = (m % 2 == 1) ? (m - 1) / 2 : m / 2 - 1;
    for (int j = 0; j < m; ++j) {
      const double xr = (double)(i - j * g) / n;
      double w = 1.0;
      for (int kk = 1; kk <= K; ++kk) w += 2.0 * cospi(2.0 * kk * xr);
      if (m % 2 == 0) w += cospi((double)m * xr);
      Wt[(long long)j * n + i] = w / m;
    }
    return;
  }
  const int np = (kind == RPA_INTERP_TRILINEAR) ? 2 : 4;
  int c = 0;
  while (c + 1 < m && nodes[c + 1] <= i) ++c;  // nodes[c] <= i
  int cols[4];
  double xs[4];
  int cnt;
  if (bc == RPA_PERIODIC) {
    cnt = np;
    const int first = c - (np / 2 - 1);
    for (int t = 0; t < np; ++t) {
      const int kk = first + t;
      const int q = ((kk % m) + m) % m;
      const int wraps = (kk - q) / m;
      cols[t] = q;
      xs[t] = (double)nodes[q] + (double)n * wraps;
    }
  } else {
    if (c > m - 2) c = m - 2;
    cnt = np < m ? np : m;
    int first = c - (cnt / 2 - 1);
    if (first < 0) first = 0;
    if (first > m - cnt) first = m - cnt;
    for (int t = 0; t < cnt; ++t) {
      cols[t] = first + t;
      xs[t] = (double)nodes[first + t];
    }
  }
  for (int t = 0; t < cnt; ++t) {
    double w = 1.0;
    for (int u = 0; u < cnt; ++u)
      if (u != t) w *= ((double)i - xs[u]) / (xs[t] - xs[u]);
    Wt[(long long)cols[t] * n + i] += w;
  }
}

cudaError_t interp_matrix(int n, int m, int bc, int kind, const long long* nodes, double* Wt,
                          cudaStream_t s) {
  k_interp_matrix<<<(n + 127) / 128, 128, 0, s>>>(n, m, bc, kind, nodes, Wt);
  note_launch();
  return cudaGetLastError();
}

// E_c = 1/(2 pi) sum_k w_k sum_j dfine[k][j]  (two deterministic reduction levels)
__global__ void k_ec_partial(long long nd, int nw, const double* __restrict__ dfine,
                             const double* __restrict__ weight, double* __restrict__ part) {
  const int k = blockIdx.y;
  double acc = 0.0;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < nd;
       p += (long long)gridDim.x * blockDim.x)
    acc += dfine[(long long)k * nd + p];
  __shared__ double sh[32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    part[(long long)k * gridDim.x + blockIdx.x] = t * weight[k];
  }
}

__global__ void k_ec_final(int n, const double* __restrict__ part, double* __restrict__ ec) {
  if (threadIdx.x != 0) return;
  double t = 0.0;
  for (int i = 0; i < n; ++i) t += part[i];
  ec[0] = t / (2.0 * 3.14159265358979323846);
}

cudaError_t ec_reduce(long long nd, int nw, const double* dfine, const double* weight,
                      double* part, int nblk, double* ec, cudaStream_t s) {
  dim3 g(nblk, nw);
  k_ec_partial<<<g, 256, 0, s>>>(nd, nw, dfine, weight, part);
  k_ec_final<<<1, 32, 0, s>>>(nblk * nw, part, ec);
  note_launch(2);
  return cudaGetLastError();
}

// scale(p) = sqrt(4 pi / -(lx + ly + lz)), zero on the null space of the Laplacian
__global__ void k_nu_scale(const double* __restrict__ l0, const double* __restrict__ l1,
                           const double* __restrict__ l2, int nx, int ny, int nz, double lmax,
                           double* __restrict__ s64, float* __restrict__ s32) {
  const long long nd = (long long)nx * ny * nz;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < nd;
       p += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(p % nx);
    const int j = (int)((p / nx) % ny);
    const int k = (int)(p / ((long long)nx * ny));
    const double neg = -(l0[i] + l1[j] + l2[k]);
    const double sc = (neg > 1e-10 * lmax) ? sqrt(4.0 * 3.14159265358979323846 / neg) : 0.0;
    s64[p] = sc;
    s32[p] = (float)sc;
  }
}

cudaError_t nu_scale(const double* l0, const double* l1, const double* l2, int nx, int ny, int nz,
                     double lmax, double* s64, float* s32, cudaStream_t s) {
  const long long nd = (long long)nx * ny * nz;
  k_nu_scale<<<(unsigned)std::min<long long>((nd + 255) / 256, 2048), 256, 0, s>>>(
      l0, l1, l2, nx, ny, nz, lmax, s64, s32);
  note_launch();
  return cudaGetLastError();
}

// Lanczos bookkeeping ----------------------------------------------------------------------
// After alpha_k = q_k^T v: store it and set coef = [beta_{k-1}, alpha_k] for the
// three-term recurrence v -= alpha_k q_k + beta_{k-1} q_{k-1}.
__global__ void k_lanczos_alpha(int nb, int k, int nl, const double* __restrict__ dots,
                                const int* __restrict__ active, double* __restrict__ alpha,
                                const double* __restrict__ beta, double* __restrict__ coef) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb || !active[b]) return;
  const double a = dots[b];
  alpha[(long long)b * nl + k] = a;
  coef[(long long)b * 2 + 0] = (k > 0) ? beta[(long long)b * nl + k - 1] : 0.0;
  coef[(long long)b * 2 + 1] = a;
}

// After ||v||^2: store beta_k, decide breakdown / early exit, write q_{k+1} scale factor.
// lstate per probe: [0] d_prev, [1] d_cur, [2] 1/beta;  steps[b] = k + 1
__global__ void k_lanczos_beta(int nb, int k, int nl, const double* __restrict__ vnorm2,
                               int* __restrict__ active, double* __restrict__ alpha,
                               double* __restrict__ beta, int* __restrict__ steps,
                               double* __restrict__ lstate, double lrtol, int fkind,
                               int* __restrict__ flags) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb || !active[b]) return;
  steps[b] = k + 1;
  double* ls = lstate + (long long)b * 4;
  const double a0 = alpha[(long long)b * nl];
  if (!isfinite(alpha[(long long)b * nl + k])) {
    active[b] = 0;
    atomicOr(flags, 1);
    return;
  }
  if (lrtol > 0.0) {
    // d^{(k)} from the current T_{k+1}
    const int kk = k + 1;
    double a[kMaxLanczos], e[kMaxLanczos], z[kMaxLanczos];
    for (int j = 0; j < kk; ++j) {
      a[j] = alpha[(long long)b * nl + j];
      e[j] = (j + 1 < kk) ? beta[(long long)b * nl + j] : 0.0;
    }
    double d = 0.0;
    if (tridiag_qr(kk, a, e, z))
      for (int j = 0; j < kk; ++j) d += z[j] * z[j] * fapply(a[j], fkind);
    const double dprev = ls[1];
    ls[1] = d;
    if (k >= 1 && fabs(d - dprev) <= lrtol * fabs(d)) {
      active[b] = 0;
      return;
    }
  }
  if (k < nl - 1) {
    const double bn = sqrt(vnorm2[b]);
    if (!isfinite(bn)) {
      active[b] = 0;
      atomicOr(flags, 1);
      return;
    }
    if (bn <= 1e-14 * fabs(a0) || bn == 0.0) {
      active[b] = 0;
      return;
    }
    beta[(long long)b * nl + k] = bn;
    ls[2] = 1.0 / bn;
  } else {
    active[b] = 0;
  }
}

// q_{k+1} = v / beta_k
__global__ void k_lanczos_next(long long nd, int k, int nl, const int* __restrict__ active,
                               const double* __restrict__ lstate, const double* __restrict__ beta,
                               const double* __restrict__ v, double* __restrict__ Q,
                               long long ldq) {
  const int b = blockIdx.y;
  if (!active[b]) return;
  const double bn = beta[(long long)b * nl + k];
  double* q = Q + (long long)b * ldq + (long long)(k + 1) * nd;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < nd;
       p += (long long)gridDim.x * blockDim.x)
    q[p] = v[(long long)b * nd + p] / bn;
}

// Q[b][0] = e_{probe_b}
__global__ void k_lanczos_start(long long nd, int nb, const long long* __restrict__ probe,
                                double* __restrict__ Q, long long ldq) {
  const int b = blockIdx.y;
  double* q = Q + (long long)b * ldq;
  const long long j = probe[b];
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < nd;
       p += (long long)gridDim.x * blockDim.x)
    q[p] = (p == j) ? 1.0 : 0.0;
}

cudaError_t lanczos_alpha(int nb, int k, int nl, const double* dots, const int* active,
                          double* alpha, const double* beta, double* coef, cudaStream_t s) {
  k_lanczos_alpha<<<(nb + 63) / 64, 64, 0, s>>>(nb, k, nl, dots, active, alpha, beta, coef);
  note_launch();
  return cudaGetLastError();
}
cudaError_t lanczos_beta(int nb, int k, int nl, const double* vnorm2, int* active, double* alpha,
                         double* beta, int* steps, double* lstate, double lrtol, int fkind,
                         int* flags, cudaStream_t s) {
  k_lanczos_beta<<<(nb + 31) / 32, 32, 0, s>>>(nb, k, nl, vnorm2, active, alpha, beta, steps,
                                               lstate, lrtol, fkind, flags);
  note_launch();
  return cudaGetLastError();
}
cudaError_t lanczos_next(long long nd, int nb, int k, int nl, const int* active,
                         const double* lstate, const double* beta, const double* v, double* Q,
                         long long ldq, cudaStream_t s) {
  dim3 g((unsigned)std::min<long long>((nd + 255) / 256, 512), nb);
  k_lanczos_next<<<g, 256, 0, s>>>(nd, k, nl, active, lstate, beta, v, Q, ldq);
  note_launch();
  return cudaGetLastError();
}
cudaError_t lanczos_start(long long nd, int nb, const long long* probe, double* Q, long long ldq,
                          cudaStream_t s) {
  dim3 g((unsigned)std::min<long long>((nd + 255) / 256, 512), nb);
  k_lanczos_start<<<g, 256, 0, s>>>(nd, nb, probe, Q, ldq);
  note_launch();
  return cudaGetLastError();
}

}  // namespace rpa
