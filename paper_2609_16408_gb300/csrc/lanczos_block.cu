// Block Lanczos quadrature (the block variant of the Lanczos quadrature of Section 3.1 that
// Section 6 names as future work): the b probes of a block (same frequency, distinct grid
// points) share one block Krylov recurrence started from [e_j1 ... e_jb].  Per block step the
// matrix-vector products are the usual per-slot ones (nu^{1/2}, Sternheimer solves, nu^{1/2});
// these kernels do the block part in FP64:
//   k_bdot / k_bdot_reduce   D[s][t, j] = Q_{t,j}^T v_s for the members t of s's block
//   k_baxpy                  v_s -= sum_{t,j} D[s][t, j] Q_{t,j}   (Gram-Schmidt pass)
//   k_bstore_a               diagonal block A_k from the first pass
//   k_bchol                  Cholesky of the block Gram matrix (Cholesky QR, applied twice),
//                            sub-diagonal block B_k = R2 R1, breakdown test
//   k_bscale                 v <- v R^{-1} (in place, or into the next basis block)
//   k_bassemble, jacobi, k_bquad   T_k, its eigen-decomposition, d_ji = [E1^T f(T) E1]_ii
// Slots of one block are consecutive; blocks hold at most kMaxBlock slots.
#include <cuda_runtime.h>

#include <cmath>

#include "cocg.cuh"

namespace rpa {

namespace {

constexpr int kMaxBlock = 8;

// D partials: grid (nchunk, slot, t*nj + j)
__global__ void __launch_bounds__(256)
    k_bdot(long long nd, const int* __restrict__ bfirst, const int* __restrict__ bsize,
           const double* __restrict__ Q, long long ldq, long long ldj, int j0, int nj,
           const double* __restrict__ V, const int* __restrict__ active, int nchunk,
           double* __restrict__ part) {
  const int c = blockIdx.x, s = blockIdx.y, tj = blockIdx.z;
  const int t = tj / nj, j = j0 + tj % nj;
  const long long slot_ld = (long long)gridDim.z;
  double acc = 0.0;
  if ((!active || active[s]) && t < bsize[s]) {
    const long long chunk_len = (nd + nchunk - 1) / nchunk;
    const long long r0 = (long long)c * chunk_len, r1 = min(r0 + chunk_len, nd);
    const double* q = Q + (long long)(bfirst[s] + t) * ldq + (long long)j * ldj;
    const double* v = V + (long long)s * nd;
    for (long long r = r0 + threadIdx.x; r < r1; r += blockDim.x) acc += q[r] * v[r];
  }
  __shared__ double sh[8];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += sh[w];
    part[((long long)s * slot_ld + tj) * nchunk + c] = tot;
  }
}

__global__ void k_bdot_reduce(int nslot, int ntj, int nchunk, const double* __restrict__ part,
                              double* __restrict__ D) {
  const int s = blockIdx.x;
  for (int tj = threadIdx.x; tj < ntj; tj += blockDim.x) {
    double tot = 0.0;
    for (int c = 0; c < nchunk; ++c) tot += part[((long long)s * ntj + tj) * nchunk + c];
    D[(long long)s * ntj + tj] = tot;
  }
}

__global__ void __launch_bounds__(256)
    k_baxpy(long long nd, const int* __restrict__ bfirst, const int* __restrict__ bsize,
            const double* __restrict__ Q, long long ldq, int nj, const double* __restrict__ D,
            int ldD, double* __restrict__ V, const int* __restrict__ active) {
  const int s = blockIdx.y;
  if (active && !active[s]) return;
  const int f = bfirst[s], nbk = bsize[s];
  const double* ds = D + (long long)s * ldD;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < nd;
       r += (long long)gridDim.x * blockDim.x) {
    double v = V[(long long)s * nd + r];
    for (int t = 0; t < nbk; ++t) {
      const double* q = Q + (long long)(f + t) * ldq + r;
      for (int j = 0; j < nj; ++j) v -= ds[t * nj + j] * q[(long long)j * nd];
    }
    V[(long long)s * nd + r] = v;
  }
}

// A_k[l][t] = D[first + l][t * nj + nj - 1] (projection on the current block; D rows ldD)
__global__ void k_bstore_a(int nblk, const int* __restrict__ bstart, const int* __restrict__ bsz,
                           const double* __restrict__ D, int ldD, int nj, int k, int nl,
                           double* __restrict__ Ab, const int* __restrict__ active) {
  const int B = blockIdx.x;
  const int f = bstart[B], n = bsz[B];
  if (active && !active[f]) return;
  double* a = Ab + ((long long)B * nl + k) * kMaxBlock * kMaxBlock;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int l = e / n, t = e % n;
    a[l * kMaxBlock + t] = D[(long long)(f + l) * ldD + t * nj + nj - 1];
  }
}

// Cholesky G = R^T R of the block Gram matrix G[l][t] = v_t^T v_l (from k_bdot, nj = 1), and
// R^{-1}.  pass 0 keeps R in Rk; pass 1 writes B_k = R R_0 to Bb.  A pivot below
// 1e-14 max|A_0| ends the block: its members become inactive and steps = k + 1.
__global__ void k_bchol(int nblk, const int* __restrict__ bstart, const int* __restrict__ bsz,
                        const double* __restrict__ G, int ldG, int pass, int k, int nl,
                        const double* __restrict__ Ab, double* __restrict__ Rk,
                        double* __restrict__ Rinv, double* __restrict__ Bb, int* active,
                        int* __restrict__ bsteps) {
  const int B = blockIdx.x * blockDim.x + threadIdx.x;
  if (B >= nblk) return;
  const int f = bstart[B], n = bsz[B];
  if (!active[f]) return;
  constexpr int M = kMaxBlock;
  double R[M][M], Ri[M][M];
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < M; ++j) R[i][j] = Ri[i][j] = 0.0;
  const double* a0 = Ab + (long long)B * nl * M * M;
  double scale = 0.0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) scale = fmax(scale, fabs(a0[i * M + j]));
  bool ok = true;
  for (int i = 0; i < n && ok; ++i) {
    for (int j = i; j < n; ++j) {
      // G[i][j] = v_j^T v_i = D[f + i][j]
      double sum = 0.5 * (G[(long long)(f + i) * ldG + j] + G[(long long)(f + j) * ldG + i]);
      for (int p = 0; p < i; ++p) sum -= R[p][i] * R[p][j];
      if (j == i) {
        if (!(sum > 0.0) || sqrt(sum) <= 1e-14 * scale) {
          ok = false;
          break;
        }
        R[i][i] = sqrt(sum);
      } else {
        R[i][j] = sum / R[i][i];
      }
    }
  }
  if (!ok) {
    for (int l = 0; l < n; ++l) active[f + l] = 0;
    bsteps[B] = k + 1;
    return;
  }
  // inverse of the upper triangular R
  for (int j = 0; j < n; ++j) {
    Ri[j][j] = 1.0 / R[j][j];
    for (int i = j - 1; i >= 0; --i) {
      double sum = 0.0;
      for (int p = i + 1; p <= j; ++p) sum += R[i][p] * Ri[p][j];
      Ri[i][j] = -sum / R[i][i];
    }
  }
  double* rk = Rk + (long long)B * M * M;
  double* ri = Rinv + (long long)B * M * M;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) ri[i * M + j] = Ri[i][j];
  if (pass == 0) {
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) rk[i * M + j] = R[i][j];
  } else {
    double* bk = Bb + ((long long)B * nl + k) * M * M;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        double sum = 0.0;
        for (int p = 0; p < n; ++p) sum += R[i][p] * rk[p * M + j];
        bk[i * M + j] = sum;
      }
  }
}

// out_l = sum_{t <= l} v_t Rinv[t][l] for the members of each block (out may alias v)
__global__ void __launch_bounds__(256)
    k_bscale(long long nd, int nblk, const int* __restrict__ bstart, const int* __restrict__ bsz,
             const double* __restrict__ Rinv, const double* V, double* out, long long ldo,
             const int* __restrict__ active) {
  const int B = blockIdx.y;
  const int f = bstart[B], n = bsz[B];
  if (!active[f]) return;
  constexpr int M = kMaxBlock;
  const double* ri = Rinv + (long long)B * M * M;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < nd;
       r += (long long)gridDim.x * blockDim.x) {
    double v[M];
    for (int t = 0; t < n; ++t) v[t] = V[(long long)(f + t) * nd + r];
    for (int l = 0; l < n; ++l) {
      double sum = 0.0;
      for (int t = 0; t <= l; ++t) sum += v[t] * ri[t * M + l];
      out[(long long)(f + l) * ldo + r] = sum;
    }
  }
}

// T (m x m, m = steps * n) from A_k (symmetrised) and B_k
__global__ void k_bassemble(int nblk, const int* __restrict__ bsz, const int* __restrict__ bsteps,
                            int steps_all, int nl, const double* __restrict__ Ab,
                            const double* __restrict__ Bb, double* __restrict__ T,
                            long long ldT, int* __restrict__ mdim) {
  const int B = blockIdx.x;
  const int n = bsz[B];
  const int st = bsteps[B] > 0 ? bsteps[B] : steps_all;
  const int m = st * n;
  constexpr int M = kMaxBlock;
  double* t = T + (long long)B * ldT;
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int i = e / m, j = e % m;
    const int bi = i / n, bj = j / n, li = i % n, lj = j % n;
    double v = 0.0;
    if (bi == bj) {
      const double* a = Ab + ((long long)B * nl + bi) * M * M;
      v = 0.5 * (a[li * M + lj] + a[lj * M + li]);
    } else if (bi == bj + 1) {
      v = Bb[((long long)B * nl + bj) * M * M + li * M + lj];
    } else if (bj == bi + 1) {
      v = Bb[((long long)B * nl + bi) * M * M + lj * M + li];
    }
    t[e] = v;
  }
  if (threadIdx.x == 0) mdim[B] = m;
}

__device__ __forceinline__ double fval(double x, int fkind) {
  if (fkind == 1) return x;
  if (fkind == 2) return x * x;
  return log1p(-x) + x;
}

// d of member l = sum_i W[l][i]^2 f(lam_i) (eigenvectors are the columns of W)
__global__ void k_bquad(int nblk, const int* __restrict__ bstart, const int* __restrict__ bsz,
                        const int* __restrict__ mdim, const double* __restrict__ W,
                        const double* __restrict__ lam, long long ldT, long long ldl, int fkind,
                        double* __restrict__ dout) {
  const int B = blockIdx.x;
  const int f = bstart[B], n = bsz[B], m = mdim[B];
  const double* w = W + (long long)B * ldT;
  const double* lm = lam + (long long)B * ldl;
  for (int l = threadIdx.x; l < n; l += blockDim.x) {
    double sum = 0.0;
    for (int i = 0; i < m; ++i) sum += w[l * m + i] * w[l * m + i] * fval(lm[i], fkind);
    dout[f + l] = sum;
  }
}

}  // namespace

int block_max() { return kMaxBlock; }

cudaError_t block_dot(long long nd, int nslot, int bmax, const int* bfirst, const int* bsize,
                      const double* Q, long long ldq, long long ldj, int j0, int nj,
                      const double* V, const int* active, double* part, int nchunk, double* D,
                      cudaStream_t s) {
  const dim3 grid(nchunk, nslot, bmax * nj);
  k_bdot<<<grid, 256, 0, s>>>(nd, bfirst, bsize, Q, ldq, ldj, j0, nj, V, active, nchunk, part);
  k_bdot_reduce<<<nslot, 128, 0, s>>>(nslot, bmax * nj, nchunk, part, D);
  note_launch(2);
  return cudaGetLastError();
}

cudaError_t block_axpy(long long nd, int nslot, const int* bfirst, const int* bsize,
                       const double* Q, long long ldq, int nj, const double* D, int ldD,
                       double* V, const int* active, cudaStream_t s) {
  const dim3 grid((unsigned)std::min<long long>((nd + 255) / 256, 512), nslot);
  k_baxpy<<<grid, 256, 0, s>>>(nd, bfirst, bsize, Q, ldq, nj, D, ldD, V, active);
  note_launch();
  return cudaGetLastError();
}

cudaError_t block_store_a(int nblk, const int* bstart, const int* bsz, const double* D, int ldD,
                          int nj, int k, int nl, double* Ab, const int* active, cudaStream_t s) {
  k_bstore_a<<<nblk, 64, 0, s>>>(nblk, bstart, bsz, D, ldD, nj, k, nl, Ab, active);
  note_launch();
  return cudaGetLastError();
}

cudaError_t block_chol(int nblk, const int* bstart, const int* bsz, const double* G, int ldG,
                       int pass, int k, int nl, const double* Ab, double* Rk, double* Rinv,
                       double* Bb, int* active, int* bsteps, cudaStream_t s) {
  k_bchol<<<(nblk + 63) / 64, 64, 0, s>>>(nblk, bstart, bsz, G, ldG, pass, k, nl, Ab, Rk, Rinv,
                                          Bb, active, bsteps);
  note_launch();
  return cudaGetLastError();
}

cudaError_t block_scale(long long nd, int nblk, const int* bstart, const int* bsz,
                        const double* Rinv, const double* V, double* out, long long ldo,
                        const int* active, cudaStream_t s) {
  const dim3 grid((unsigned)std::min<long long>((nd + 255) / 256, 512), nblk);
  k_bscale<<<grid, 256, 0, s>>>(nd, nblk, bstart, bsz, Rinv, V, out, ldo, active);
  note_launch();
  return cudaGetLastError();
}

cudaError_t block_quadrature(int nblk, const int* bstart, const int* bsz, const int* bsteps,
                             int steps_all, int nl, const double* Ab, const double* Bb, double* T,
                             double* W, double* lam, long long ldT, long long ldl, int* mdim,
                             int fkind, double* dout, cudaStream_t s) {
  k_bassemble<<<nblk, 256, 0, s>>>(nblk, bsz, bsteps, steps_all, nl, Ab, Bb, T, ldT, mdim);
  cudaError_t e = jacobi_eig_batched(T, W, lam, mdim, nblk, ldT, ldl, s);
  if (e != cudaSuccess) return e;
  k_bquad<<<nblk, 32, 0, s>>>(nblk, bstart, bsz, mdim, W, lam, ldT, ldl, fkind, dout);
  note_launch(2);
  return cudaGetLastError();
}

}  // namespace rpa
