// Small dense contractions on the path: the Galerkin projection over the occupied space
// (Section 4), mode products for nu^{1/2} (Kronecker-product formalism, Section 4) and for
// the separable interpolation operators (Section 3.2), Lanczos dot products and combinations
// (Section 3.1, Algorithm 1), and the 1-D eigen-decompositions behind nu^{1/2}.
#include <cuda_runtime.h>

#include "cocg.cuh"

namespace rpa {

// -------------------------------------------------------------------------------------------
// Galerkin projection
// -------------------------------------------------------------------------------------------
// gpart[b][c][k][n] = sum_{r in chunk c} psi_k(r) psi_n(r) u_b(r)
template <typename T>
__global__ void __launch_bounds__(256) k_gram(long long nd, int ns, const T* __restrict__ psi,
                                              const T* __restrict__ u,
                                              const int* __restrict__ active, int nchunk,
                                              long long chunk_len, double* __restrict__ gpart) {
  constexpr int TS = 32, RK = 32;
  __shared__ T sA[RK][TS + 1];
  __shared__ T sB[RK][TS + 1];
  const int nt = (ns + TS - 1) / TS;
  const int kt = blockIdx.x / nt, ntl = blockIdx.x - kt * nt;
  const int b = blockIdx.y, c = blockIdx.z;
  if (active && !active[b]) return;
  const int k0 = kt * TS, n0 = ntl * TS;
  const long long r0 = (long long)c * chunk_len;
  const long long r1 = min(r0 + chunk_len, nd);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const T* ub = u + (long long)b * nd;
  T acc[2][2] = {{0, 0}, {0, 0}};
  for (long long rb = r0; rb < r1; rb += RK) {
    for (int e = threadIdx.x; e < RK * TS; e += 256) {
      const int kk = e / RK, rr = e - kk * RK;
      const long long r = rb + rr;
      const bool okr = r < r1;
      const int k = k0 + kk, n = n0 + kk;
      sA[rr][kk] = (okr && k < ns) ? psi[(long long)k * nd + r] : (T)0;
      sB[rr][kk] = (okr && n < ns) ? psi[(long long)n * nd + r] * ub[r] : (T)0;
    }
    __syncthreads();
#pragma unroll 8
    for (int rr = 0; rr < RK; ++rr) {
      const T a0 = sA[rr][2 * ty], a1 = sA[rr][2 * ty + 1];
      const T b0 = sB[rr][2 * tx], b1 = sB[rr][2 * tx + 1];
      acc[0][0] += a0 * b0;
      acc[0][1] += a0 * b1;
      acc[1][0] += a1 * b0;
      acc[1][1] += a1 * b1;
    }
    __syncthreads();
  }
  double* out = gpart + ((long long)b * nchunk + c) * ns * ns;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int k = k0 + 2 * ty + i, n = n0 + 2 * tx + j;
      if (k < ns && n < ns) out[(long long)k * ns + n] = (double)acc[i][j];
    }
}

// C_b[k][n] = (-dV sum_c gpart) / (eps_k - eps_n - i w_b)
template <typename T>
__global__ void k_gram_coef(int ns, int nchunk, const double* __restrict__ gpart,
                            const double* __restrict__ eps, const double* __restrict__ omega,
                            const int* __restrict__ active, double dV, cpx<T>* __restrict__ cmat) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ns * ns) return;
  const int k = e / ns, n = e - k * ns;
  double g = 0.0;
  const double* gp = gpart + (long long)b * nchunk * ns * ns + e;
  for (int c = 0; c < nchunk; ++c) g += gp[(long long)c * ns * ns];
  g *= -dV;
  const double a = eps[k] - eps[n], w = omega[b];
  const double den = a * a + w * w;
  // g / (a - i w) = g (a + i w) / (a^2 + w^2)
  cpx<T> cv = mk<T>((T)0, (T)0);
  if (den > 0.0) cv = mk<T>((T)(g * a / den), (T)(g * w / den));
  cmat[(long long)b * ns * ns + e] = cv;
}

// x0[(b,n)][r] = sum_k psi_k(r) C_b[k][n]; output tile 64 points x 32 states for one b.
// Point tiles run along gridDim.x (up to 2^31 - 1 tiles), (b, state tile) along gridDim.y.
template <typename T>
__global__ void __launch_bounds__(256) k_x0(long long nd, int ns, int nb,
                                            const T* __restrict__ psi,
                                            const cpx<T>* __restrict__ cmat,
                                            const int* __restrict__ active,
                                            cpx<T>* __restrict__ x0) {
  constexpr int TR = 64, TN = 32, KK = 16;
  __shared__ T sP[KK][TR];
  __shared__ cpx<T> sC[KK][TN];
  const int ntn = (ns + TN - 1) / TN;
  const int b = blockIdx.y / ntn, nt = blockIdx.y - b * ntn;
  if (active && !active[b]) return;
  const long long r0 = (long long)blockIdx.x * TR;
  const int n0 = nt * TN;
  const int tr = threadIdx.x & 15, tn = threadIdx.x >> 4;  // 4 points x 2 states per thread
  cpx<T> acc[4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) acc[i][j] = mk<T>((T)0, (T)0);
  const cpx<T>* cb = cmat + (long long)b * ns * ns;
  for (int kb = 0; kb < ns; kb += KK) {
    for (int e = threadIdx.x; e < KK * TR; e += 256) {
      const int kk = e / TR, rr = e - kk * TR;
      const long long r = r0 + rr;
      sP[kk][rr] = (kb + kk < ns && r < nd) ? psi[(long long)(kb + kk) * nd + r] : (T)0;
    }
    for (int e = threadIdx.x; e < KK * TN; e += 256) {
      const int kk = e / TN, nn = e - kk * TN;
      sC[kk][nn] = (kb + kk < ns && n0 + nn < ns) ? cb[(long long)(kb + kk) * ns + n0 + nn]
                                                   : mk<T>((T)0, (T)0);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < KK; ++kk) {
      T pv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) pv[i] = sP[kk][tr + 16 * i];
      const cpx<T> c0 = sC[kk][2 * tn], c1 = sC[kk][2 * tn + 1];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        acc[i][0] = caxpy_r(acc[i][0], pv[i], c0);
        acc[i][1] = caxpy_r(acc[i][1], pv[i], c1);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const long long r = r0 + tr + 16 * i;
    if (r >= nd) continue;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int n = n0 + 2 * tn + j;
      if (n < ns) x0[((long long)b * ns + n) * nd + r] = acc[i][j];
    }
  }
}

template <typename T>
cudaError_t galerkin_guess(long long nd, int ns, int nb, const T* psi, const double* eps,
                           const double* omega, const T* u, const int* probe_active, double dV,
                           double* gpart, int nchunk, cpx<T>* cmat, cpx<T>* x0, cudaStream_t s) {
  const long long chunk_len = (nd + nchunk - 1) / nchunk;
  const int nt = (ns + 31) / 32;
  dim3 g1(nt * nt, nb, nchunk);
  k_gram<T><<<g1, 256, 0, s>>>(nd, ns, psi, u, probe_active, nchunk, chunk_len, gpart);
  dim3 g2((ns * ns + 255) / 256, nb);
  k_gram_coef<T><<<g2, 256, 0, s>>>(ns, nchunk, gpart, eps, omega, probe_active, dV, cmat);
  if ((long long)nb * ((ns + 31) / 32) > 65535) return cudaErrorInvalidValue;
  dim3 g3((unsigned)((nd + 63) / 64), nb * ((ns + 31) / 32));
  k_x0<T><<<g3, 256, 0, s>>>(nd, ns, nb, psi, cmat, probe_active, x0);
  note_launch(3);
  return cudaGetLastError();
}

template <typename T>
cudaError_t gram_coef(int ns, int nb, int nchunk, const double* gpart, const double* eps,
                      const double* omega, const int* active, double dV, cpx<T>* cmat,
                      cudaStream_t s) {
  dim3 g2((ns * ns + 255) / 256, nb);
  k_gram_coef<T><<<g2, 256, 0, s>>>(ns, nchunk, gpart, eps, omega, active, dV, cmat);
  return cudaGetLastError();
}
template cudaError_t gram_coef<float>(int, int, int, const double*, const double*, const double*,
                                      const int*, double, cpx<float>*, cudaStream_t);

// -------------------------------------------------------------------------------------------
// mode products: out[.., a, ..] = sum_i Mt[i][a] in[.., i, ..] along one axis
// -------------------------------------------------------------------------------------------
template <typename TI, typename TO, typename T>
__global__ void __launch_bounds__(256) k_mode(const TI* __restrict__ in, long long in_bs,
                                              TO* __restrict__ out, long long out_bs,
                                              const T* __restrict__ Mt, int axis, int n0, int n1,
                                              int n2, int nout, long long out_per,
                                              const T* __restrict__ scale) {
  const int b = blockIdx.y;
  const long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= out_per) return;
  int d[3] = {n0, n1, n2};
  d[axis] = nout;
  const int i0 = (int)(o % d[0]);
  const long long t = o / d[0];
  const int i1 = (int)(t % d[1]);
  const int i2 = (int)(t / d[1]);
  const int nin = (axis == 0) ? n0 : (axis == 1) ? n1 : n2;
  const int a = (axis == 0) ? i0 : (axis == 1) ? i1 : i2;
  long long base, stride;
  if (axis == 0) {
    base = (long long)n0 * (i1 + (long long)n1 * i2);
    stride = 1;
  } else if (axis == 1) {
    base = i0 + (long long)n0 * n1 * i2;
    stride = n0;
  } else {
    base = i0 + (long long)n0 * i1;
    stride = (long long)n0 * n1;
  }
  const TI* src = in + (long long)b * in_bs + base;
  T acc = 0;
  for (int i = 0; i < nin; ++i) acc += Mt[(long long)i * nout + a] * (T)src[i * stride];
  if (scale) acc *= scale[o];
  out[(long long)b * out_bs + o] = (TO)acc;
}

template <typename TI, typename TO, typename T>
cudaError_t mode_product(const TI* in, long long in_bs, TO* out, long long out_bs, const T* Mt,
                         int axis, const int* dims_in, int nout, int batch, const T* scale,
                         cudaStream_t s) {
  long long in_per = (long long)dims_in[0] * dims_in[1] * dims_in[2];
  long long out_per = in_per / dims_in[axis] * nout;
  dim3 grid((unsigned)((out_per + 255) / 256), batch);
  k_mode<TI, TO, T><<<grid, 256, 0, s>>>(in, in_bs, out, out_bs, Mt, axis, dims_in[0],
                                          dims_in[1], dims_in[2], nout, out_per, scale);
  note_launch();
  return cudaGetLastError();
}

// -------------------------------------------------------------------------------------------
// Lanczos helpers (FP64)
// -------------------------------------------------------------------------------------------
constexpr int kDotGroup = 8;

// part[b][c][m - m0] = sum_{r in chunk c} Q[b][m][r] v[b][r]
__global__ void __launch_bounds__(256) k_multi_dot(long long nd, const double* __restrict__ Q,
                                                   long long ldq, int m0, int m1,
                                                   const double* __restrict__ v,
                                                   const int* __restrict__ active, int nchunk,
                                                   double* __restrict__ part) {
  const int c = blockIdx.x, b = blockIdx.y, mg = m0 + blockIdx.z * kDotGroup;
  if (active && !active[b]) return;
  const int mm = min(kDotGroup, m1 - mg);
  const long long chunk_len = (nd + nchunk - 1) / nchunk;
  const long long r0 = (long long)c * chunk_len, r1 = min(r0 + chunk_len, nd);
  double acc[kDotGroup];
#pragma unroll
  for (int j = 0; j < kDotGroup; ++j) acc[j] = 0.0;
  const double* vb = v + (long long)b * nd;
  const double* Qb = Q + (long long)b * ldq + (long long)mg * nd;
  for (long long r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
    const double vr = vb[r];
#pragma unroll
    for (int j = 0; j < kDotGroup; ++j)
      if (j < mm) acc[j] += Qb[(long long)j * nd + r] * vr;
  }
  __shared__ double sh[8 * kDotGroup];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < kDotGroup; ++j)
    for (int o = 16; o > 0; o >>= 1) acc[j] += __shfl_down_sync(0xffffffffu, acc[j], o);
  if (lane == 0)
    for (int j = 0; j < kDotGroup; ++j) sh[wid * kDotGroup + j] = acc[j];
  __syncthreads();
  if (threadIdx.x < mm) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w * kDotGroup + threadIdx.x];
    const int nm = m1 - m0;
    part[((long long)b * nchunk + c) * nm + (mg - m0) + threadIdx.x] = t;
  }
}

__global__ void k_dot_reduce(int nb, int nm, int nchunk, const double* __restrict__ part,
                             const int* __restrict__ active, double* __restrict__ dots) {
  const int b = blockIdx.x;
  if (active && !active[b]) return;
  for (int m = threadIdx.x; m < nm; m += blockDim.x) {
    double t = 0.0;
    for (int c = 0; c < nchunk; ++c) t += part[((long long)b * nchunk + c) * nm + m];
    dots[(long long)b * nm + m] = t;
  }
}

cudaError_t multi_dot(long long nd, int nb, const double* Q, long long ldq, int m0, int m1,
                      const double* v, const int* active, double* part, int nchunk,
                      double* dots, cudaStream_t s) {
  const int nm = m1 - m0;
  dim3 grid(nchunk, nb, (nm + kDotGroup - 1) / kDotGroup);
  k_multi_dot<<<grid, 256, 0, s>>>(nd, Q, ldq, m0, m1, v, active, nchunk, part);
  k_dot_reduce<<<nb, 64, 0, s>>>(nb, nm, nchunk, part, active, dots);
  note_launch(2);
  return cudaGetLastError();
}

// v[b][r] -= sum_{m in [m0, m1)} coef[b][m - m0] Q[b][m][r]
__global__ void __launch_bounds__(256) k_multi_axpy(long long nd, const double* __restrict__ Q,
                                                    long long ldq, int m0, int m1,
                                                    const double* __restrict__ coef, int ldc,
                                                    double* __restrict__ v,
                                                    const int* __restrict__ active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const double* Qb = Q + (long long)b * ldq;
  const double* cb = coef + (long long)b * ldc;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < nd;
       r += (long long)gridDim.x * blockDim.x) {
    double t = v[(long long)b * nd + r];
    for (int m = m0; m < m1; ++m) t -= cb[m - m0] * Qb[(long long)m * nd + r];
    v[(long long)b * nd + r] = t;
  }
}

cudaError_t multi_axpy(long long nd, int nb, const double* Q, long long ldq, int m0, int m1,
                       const double* coef, int ldc, double* v, const int* active, cudaStream_t s) {
  dim3 grid((unsigned)std::min<long long>((nd + 255) / 256, 512), nb);
  k_multi_axpy<<<grid, 256, 0, s>>>(nd, Q, ldq, m0, m1, coef, ldc, v, active);
  note_launch();
  return cudaGetLastError();
}

__global__ void k_d2f(const double* __restrict__ a, float* __restrict__ b, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}
__global__ void k_f2d(const float* __restrict__ a, double* __restrict__ b, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    b[i] = (double)a[i];
}
cudaError_t convert_d2f(const double* a, float* b, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_d2f<<<(unsigned)std::min<long long>((n + 255) / 256, 4096), 256, 0, s>>>(a, b, n);
  note_launch();
  return cudaGetLastError();
}
cudaError_t convert_f2d(const float* a, double* b, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_f2d<<<(unsigned)std::min<long long>((n + 255) / 256, 4096), 256, 0, s>>>(a, b, n);
  note_launch();
  return cudaGetLastError();
}

// -------------------------------------------------------------------------------------------
// cyclic Jacobi eigen-decomposition of a small symmetric matrix (one block); a is n x n
// row-major and is overwritten; v receives eigenvectors as columns; lam the eigenvalues.
// -------------------------------------------------------------------------------------------
__device__ void jacobi_body(double* a, double* v, double* lam, int n) {
  __shared__ double s_c, s_s, s_red[32];
  __shared__ int s_skip, s_done;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) v[e] = ((e / n) == (e % n)) ? 1.0 : 0.0;
  __syncthreads();
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      const double q = a[e] * a[e];
      tot += q;
      if (e / n != e % n) off += q;
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_down_sync(0xffffffffu, off, o);
      tot += __shfl_down_sync(0xffffffffu, tot, o);
    }
    if ((threadIdx.x & 31) == 0) {
      s_red[threadIdx.x >> 5] = off;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double o2 = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) o2 += s_red[w];
      s_red[31] = o2;
    }
    __syncthreads();
    const double offall = s_red[31];
    __syncthreads();
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = tot;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t2 = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t2 += s_red[w];
      s_done = (offall <= 1e-30 * t2 || offall == 0.0) ? 1 : 0;
    }
    __syncthreads();
    if (s_done) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        if (threadIdx.x == 0) {
          const double apq = a[p * n + q];
          s_skip = (apq == 0.0);
          if (!s_skip) {
            const double th = 0.5 * atan2(2.0 * apq, a[q * n + q] - a[p * n + p]);
            s_c = cos(th);
            s_s = sin(th);
          }
        }
        __syncthreads();
        if (!s_skip) {
          const double c = s_c, sn = s_s;
          for (int k = threadIdx.x; k < n; k += blockDim.x) {
            const double akp = a[k * n + p], akq = a[k * n + q];
            a[k * n + p] = c * akp - sn * akq;
            a[k * n + q] = sn * akp + c * akq;
          }
          __syncthreads();
          for (int k = threadIdx.x; k < n; k += blockDim.x) {
            const double apk = a[p * n + k], aqk = a[q * n + k];
            a[p * n + k] = c * apk - sn * aqk;
            a[q * n + k] = sn * apk + c * aqk;
            const double vkp = v[k * n + p], vkq = v[k * n + q];
            v[k * n + p] = c * vkp - sn * vkq;
            v[k * n + q] = sn * vkp + c * vkq;
          }
        }
        __syncthreads();
      }
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) lam[i] = a[i * n + i];
}

__global__ void k_jacobi(double* a, double* v, double* lam, int n) { jacobi_body(a, v, lam, n); }

// one matrix per block: matrix b of order n[b] at a + b * lda (eigenvectors likewise), its
// eigenvalues at lam + b * ldl
__global__ void k_jacobi_batched(double* a, double* v, double* lam, const int* n, long long lda,
                                 long long ldl) {
  const long long b = blockIdx.x;
  jacobi_body(a + b * lda, v + b * lda, lam + b * ldl, n[b]);
}

cudaError_t jacobi_eig_batched(double* a, double* v, double* lam, const int* n, int count,
                               long long lda, long long ldl, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_jacobi_batched<<<count, 256, 0, s>>>(a, v, lam, n, lda, ldl);
  note_launch();
  return cudaGetLastError();
}

cudaError_t jacobi_eig(double* a, double* v, double* lam, int n, cudaStream_t s) {
  k_jacobi<<<1, 256, 0, s>>>(a, v, lam, n);
  note_launch();
  return cudaGetLastError();
}

template cudaError_t galerkin_guess<double>(long long, int, int, const double*, const double*,
                                            const double*, const double*, const int*, double,
                                            double*, int, cpx<double>*, cpx<double>*,
                                            cudaStream_t);
template cudaError_t galerkin_guess<float>(long long, int, int, const float*, const double*,
                                           const double*, const float*, const int*, double,
                                           double*, int, cpx<float>*, cpx<float>*, cudaStream_t);
#define RPA_MODE_INST(TI, TO, T)                                                              \
  template cudaError_t mode_product<TI, TO, T>(const TI*, long long, TO*, long long, const T*, \
                                                int, const int*, int, int, const T*, cudaStream_t);
RPA_MODE_INST(double, double, double)
RPA_MODE_INST(double, float, float)
RPA_MODE_INST(float, float, float)
RPA_MODE_INST(float, double, float)
#undef RPA_MODE_INST

}  // namespace rpa
