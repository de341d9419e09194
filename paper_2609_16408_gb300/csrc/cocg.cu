// Batched Sternheimer solves by COCG (Eq. 4, Section 4) with the finite-difference
// Hamiltonian stencil, local potential and nonlocal projectors.
//
// A batch holds S = B x N_s complex-symmetric systems (H - eps_n - i w_b) x = b,
// b = -psi_n (.) u_b.  Every vector is S x N_d complex (interleaved).  Kernels are launched
// over (tiles, systems); a system whose status is not selected returns at once, so converged
// systems retire individually.  Reductions are deterministic: each block writes its partial
// sums, and one warp per system adds them in a fixed order.
#include <cuda_runtime.h>

#include "cocg.cuh"
#include "fused_dev.cuh"

namespace rpa {

// -------------------------------------------------------------------------------------------
// helpers
// -------------------------------------------------------------------------------------------
__device__ __forceinline__ int wrap_index(int j, int n, int bc) {
  if (bc == 0) {
    while (j < 0) j += n;
    while (j >= n) j -= n;
    return j;
  }
  return (j < 0 || j >= n) ? -1 : j;
}

// (-1/2 Lap_h + V - sigma) x at one point, plus the nonlocal term from precomputed
// projector coefficients cd (gamma dV chi^T x per internal group and projector).
template <typename T>
__device__ __forceinline__ cpx<T> h_at(const Stencil<T>& st, const T* __restrict__ vloc,
                                       const NonlocalDev<T>& nl, const cpx<T>* __restrict__ x,
                                       const cpx<T>* __restrict__ cd, int ix, int iy, int iz,
                                       long long p, cpx<T> sigma) {
  const cpx<T> xc = x[p];
  const T dg = st.c0 + vloc[p];
  cpx<T> acc = mk<T>(dg * xc.re - (sigma.re * xc.re - sigma.im * xc.im),
                     dg * xc.im - (sigma.re * xc.im + sigma.im * xc.re));
  const long long sx = 1, sy = st.nx, sz = (long long)st.nx * st.ny;
  const long long base = p - ix * sx - iy * sy - iz * sz;
#pragma unroll 4
  for (int m = 1; m <= st.R; ++m) {
    int a = wrap_index(ix + m, st.nx, st.bcx), b = wrap_index(ix - m, st.nx, st.bcx);
    cpx<T> s = mk<T>(0, 0);
    if (a >= 0) s = cadd(s, x[base + a * sx + iy * sy + iz * sz]);
    if (b >= 0) s = cadd(s, x[base + b * sx + iy * sy + iz * sz]);
    acc = caxpy_r(acc, st.cx[m], s);
    a = wrap_index(iy + m, st.ny, st.bcy);
    b = wrap_index(iy - m, st.ny, st.bcy);
    s = mk<T>(0, 0);
    if (a >= 0) s = cadd(s, x[base + ix * sx + a * sy + iz * sz]);
    if (b >= 0) s = cadd(s, x[base + ix * sx + b * sy + iz * sz]);
    acc = caxpy_r(acc, st.cy[m], s);
    a = wrap_index(iz + m, st.nz, st.bcz);
    b = wrap_index(iz - m, st.nz, st.bcz);
    s = mk<T>(0, 0);
    if (a >= 0) s = cadd(s, x[base + ix * sx + iy * sy + a * sz]);
    if (b >= 0) s = cadd(s, x[base + ix * sx + iy * sy + b * sz]);
    acc = caxpy_r(acc, st.cz[m], s);
  }
  if (nl.ngroup > 0) {
    const int e0 = nl.p_off[p], e1 = nl.p_off[p + 1];
    for (int e = e0; e < e1; ++e) {
      const int g = nl.p_grp[e];
      const T* ch = nl.p_chi + (long long)e * kProjChunk;
      const cpx<T>* c = cd + (long long)g * kProjChunk;
#pragma unroll
      for (int l = 0; l < kProjChunk; ++l) acc = caxpy_r(acc, ch[l], c[l]);
    }
  }
  return acc;
}

template <typename T>
__device__ __forceinline__ void point_coords(long long p, const Stencil<T>& st, int& ix, int& iy,
                                             int& iz) {
  const long long pl = (long long)st.nx * st.ny;
  iz = (int)(p / pl);
  const long long rem = p - (long long)iz * pl;
  iy = (int)(rem / st.nx);
  ix = (int)(rem - (long long)iy * st.nx);
}

// Block reduction of NQ values; thread 0 returns the totals.
template <typename A, int NQ>
__device__ __forceinline__ void block_reduce_t(A (&v)[NQ], A* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
  }
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) sh[wid * NQ + q] = v[q];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < nw; ++w) {
#pragma unroll
      for (int q = 0; q < NQ; ++q) v[q] += sh[w * NQ + q];
    }
  }
}

template <int NQ>
__device__ __forceinline__ void block_reduce(double (&v)[NQ], double* sh) {
  block_reduce_t<double, NQ>(v, sh);
}
__device__ __forceinline__ int status_of(const int* sysi, int s) {
  return sysi[(long long)s * kSysI + kStatus];
}
__device__ __forceinline__ bool selected(const int* sysi, int s, int mask) {
  return (mask >> status_of(sysi, s)) & 1;
}

// -------------------------------------------------------------------------------------------
// projector dot products: cd[s][g][l] = gamma_{g,l} dV sum_e chi_{g,l}(e) v_s(idx_e)
// -------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(128) k_proj_dots(NonlocalDev<T> nl, long long nd,
                                                   const cpx<T>* __restrict__ vec,
                                                   const int* __restrict__ sysi, int mask,
                                                   cpx<T>* __restrict__ cd) {
  const int g = blockIdx.x, s = blockIdx.y;
  if (sysi && !selected(sysi, s, mask)) return;
  // sums in the working precision: a thread adds a few dozen entries, so FP32 keeps ~1e-6
  // relative accuracy in the FP32 path without the 1/58-rate FP64 adds
  __shared__ T sh[4 * 2 * kProjChunk];
  const cpx<T>* v = vec + (long long)s * nd;
  T acc[2 * kProjChunk];
#pragma unroll
  for (int q = 0; q < 2 * kProjChunk; ++q) acc[q] = (T)0;
  for (int e = nl.g_off[g] + threadIdx.x; e < nl.g_off[g + 1]; e += blockDim.x) {
    const cpx<T> xv = v[nl.g_idx[e]];
    const T* ch = nl.g_chi + (long long)e * kProjChunk;
#pragma unroll
    for (int l = 0; l < kProjChunk; ++l) {
      acc[2 * l] += ch[l] * xv.re;
      acc[2 * l + 1] += ch[l] * xv.im;
    }
  }
  block_reduce_t<T, 2 * kProjChunk>(acc, sh);
  if (threadIdx.x == 0) {
    cpx<T>* out = cd + ((long long)s * nl.ngroup + g) * kProjChunk;
#pragma unroll
    for (int l = 0; l < kProjChunk; ++l) {
      const T c = nl.coef[g * kProjChunk + l];
      out[l] = mk<T>(c * acc[2 * l], c * acc[2 * l + 1]);
    }
  }
}

// -------------------------------------------------------------------------------------------
// y = (H - sigma) x for independent vectors (step check of the H apply)
// -------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_apply_h(Stencil<T> st, const T* __restrict__ vloc,
                                                 NonlocalDev<T> nl, long long nd,
                                                 const cpx<T>* __restrict__ x,
                                                 const cpx<T>* __restrict__ sigma,
                                                 const cpx<T>* __restrict__ cd,
                                                 cpx<T>* __restrict__ y) {
  const int s = blockIdx.y;
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nd) return;
  int ix, iy, iz;
  point_coords(p, st, ix, iy, iz);
  y[(long long)s * nd + p] = h_at(st, vloc, nl, x + (long long)s * nd,
                                  cd + (long long)s * nl.ngroup * kProjChunk, ix, iy, iz, p,
                                  sigma[s]);
}

// -------------------------------------------------------------------------------------------
// COCG kernels (the true residual r = b - A x is in cocg_resid.cu)
// -------------------------------------------------------------------------------------------
// per-system scalar steps (one warp per system, partial sums added in tile order)
// -------------------------------------------------------------------------------------------
__device__ __forceinline__ void warp_sum_tiles(const double* part, int tiles, int lane,
                                               double (&v)[4]) {
  for (int q = 0; q < 4; ++q) v[q] = 0.0;
  for (int t = lane; t < tiles; t += 32)
    for (int q = 0; q < 4; ++q) v[q] += part[(long long)t * 4 + q];
  for (int q = 0; q < 4; ++q)
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
}

__device__ __forceinline__ void cdiv(double ar, double ai, double br, double bi, double& qr,
                                     double& qi) {
  const double den = br * br + bi * bi;
  qr = (ar * br + ai * bi) / den;
  qi = (ai * br - ar * bi) / den;
}

// kind: 0 init after the first residual (target = tol ||b||, or round target for
//        refinement), 1 alpha, 2 beta/convergence, 3 true-residual recheck,
//        4 refinement check (FP64 residual of the mixed form)
__global__ void k_scalars(int nsys, int tiles, int stride, const double* __restrict__ part,
                          double* sysd, int* sysi, int kind, int mask, double tol,
                          double inner_tol, int maxit, int max_restart,
                          const int* __restrict__ list) {
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= nsys) return;
  const int s = list ? list[i] : i;
  if (s < 0) return;  // past the active count of a graph launch
  int* si = sysi + (long long)s * kSysI;
  double* sd = sysd + (long long)s * kSysD;
  const int st = si[kStatus];
  if (!((mask >> st) & 1)) return;
  double v[4];
  warp_sum_tiles(part + (long long)s * stride * 4, tiles, lane, v);
  if (lane != 0) return;
  if (kind == 0 || kind == 5) {
    sd[kNlDot] = 0.0;
    sd[kNlDot + 1] = 0.0;
  }
  if (kind == 0) {  // after r0 = b - A x0
    const double rn = sqrt(v[0]), bn = sqrt(v[1]);
    sd[kBnorm] = bn;
    sd[kRnorm] = rn;
    sd[kTarget] = tol * bn;
    sd[kRho] = v[2];
    sd[kRho + 1] = v[3];
    si[kIters] = 0;
    si[kRestarts] = 0;
    si[kIterBase] = 0;
    si[kStatus] = (bn == 0.0 || rn <= tol * bn) ? kFinal : kActive;
    if (!isfinite(rn) || !isfinite(bn)) si[kStatus] = kBreakdown;
  } else if (kind == 1) {  // alpha = rho / (p^T A p)
    if (si[kIters] >= maxit) {
      si[kStatus] = kMaxit;
      return;
    }
    v[0] += sd[kNlDot];
    v[1] += sd[kNlDot + 1];
    double ar, ai;
    if ((v[0] == 0.0 && v[1] == 0.0) || !isfinite(v[0]) || !isfinite(v[1])) {
      si[kStatus] = kBreakdown;
      return;
    }
    cdiv(sd[kRho], sd[kRho + 1], v[0], v[1], ar, ai);
    sd[kAlpha] = ar;
    sd[kAlpha + 1] = ai;
  } else if (kind == 2) {  // after the update: convergence test, beta
    const double rn = sqrt(v[0]);
    si[kIters] += 1;
    sd[kRnorm] = rn;
    if (!isfinite(rn)) {
      si[kStatus] = kBreakdown;
      return;
    }
    if (rn <= sd[kTarget]) {
      si[kStatus] = kConverged;
      return;
    }
    double br, bi;
    cdiv(v[2], v[3], sd[kRho], sd[kRho + 1], br, bi);
    sd[kBeta] = br;
    sd[kBeta + 1] = bi;
    sd[kRho] = v[2];
    sd[kRho + 1] = v[3];
  } else if (kind == 3) {  // true residual of a recursively converged system
    const double rn = sqrt(v[0]);
    sd[kRnormTrue] = rn;
    if (rn <= sd[kTarget]) {
      si[kStatus] = kFinal;
    } else if (si[kRestarts] >= max_restart || !isfinite(rn)) {
      // the restarts are used up and the true residual still misses the tolerance
      si[kStatus] = isfinite(rn) ? kMaxit : kBreakdown;
    } else {
      si[kRestarts] += 1;
      sd[kRho] = v[2];
      sd[kRho + 1] = v[3];
      si[kStatus] = (si[kIters] >= maxit) ? kMaxit : kActive;
    }
  } else if (kind == 4 || kind == 6) {  // mixed form: FP64 residual of the FP64 iterate
    const double rn = sqrt(v[0]);
    sd[kRnormTrue] = rn;
    if (rn <= tol * sd[kBnorm] || !isfinite(rn)) {
      si[kStatus] = isfinite(rn) ? kFinal : kBreakdown;
    } else {
      // correction round: solve A d = r in low precision from d = 0.  kind 4 restarts the
      // recurrence (p = r); kind 6 keeps the previous direction and continues it with the
      // true residual in place of the recursive one: beta = rho_new / rho_k, where rho_k
      // (still in sysd) belongs to the residual that formed the last direction.  When the
      // true residual has drifted far above the recursive one (|beta| > 4: the low-precision
      // recurrence went below what its rounding can resolve), the old direction no longer
      // fits the new residual and the round restarts instead (beta = 0, p = r).
      sd[kTarget] = fmax(inner_tol * rn, 0.5 * tol * sd[kBnorm]);
      double br = 0.0, bi = 0.0;
      if (kind == 6 && si[kIters] > si[kIterBase])
        cdiv(v[2], v[3], sd[kRho], sd[kRho + 1], br, bi);
      if (!isfinite(br) || !isfinite(bi) || br * br + bi * bi > 16.0) br = bi = 0.0;
      sd[kBeta] = br;
      sd[kBeta + 1] = bi;
      sd[kRho] = v[2];
      sd[kRho + 1] = v[3];
      si[kIterBase] = si[kIters];
      si[kStatus] = (si[kIters] >= maxit) ? kMaxit : kActive;
      si[kRestarts] += 1;
    }
  } else if (kind == 7) {  // mixed form, after the last refinement round: final FP64 check
    const double rn = sqrt(v[0]);
    sd[kRnormTrue] = rn;
    si[kStatus] = !isfinite(rn) ? kBreakdown : (rn <= tol * sd[kBnorm] ? kFinal : kMaxit);
  } else if (kind == 5) {  // mixed form init: low-precision round 0 target
    const double rn = sqrt(v[0]), bn = sqrt(v[1]);
    sd[kBnorm] = bn;
    sd[kRnorm] = rn;
    sd[kTarget] = inner_tol * bn;
    sd[kRho] = v[2];
    sd[kRho + 1] = v[3];
    si[kIters] = 0;
    si[kRestarts] = 0;
    si[kIterBase] = 0;
    si[kStatus] = (bn == 0.0 || rn <= inner_tol * bn) ? kConverged : kActive;
    if (!isfinite(rn) || !isfinite(bn)) si[kStatus] = kBreakdown;
  }
}

// counts of systems per status
__global__ void k_count_status(int nsys, const int* __restrict__ sysi, int* __restrict__ counts,
                               int* __restrict__ list) {
  __shared__ int sc[kNumStatus];
  if (threadIdx.x < kNumStatus) sc[threadIdx.x] = 0;
  __syncthreads();
  for (int s = threadIdx.x; s < nsys; s += blockDim.x) {
    const int st = sysi[(long long)s * kSysI + kStatus];
    const int pos = atomicAdd(&sc[st], 1);
    if (list && st == kActive) list[pos] = s;
  }
  __syncthreads();
  if (threadIdx.x < kNumStatus) counts[threadIdx.x] = sc[threadIdx.x];
  // entries past the active count are -1: launches sized above the count skip them
  if (list)
    for (int i = sc[kActive] + threadIdx.x; i < nsys; i += blockDim.x) list[i] = -1;
}

__global__ void k_loop_cond(const int* __restrict__ counts, unsigned long long* __restrict__ ctl,
                            cudaGraphConditionalHandle h, int wnext, int limit, int add_iters,
                            int add_launches) {
  const unsigned long long it = ctl[0] + (unsigned long long)add_iters;
  ctl[0] = it;
  ctl[1] += (unsigned long long)add_launches;
  cudaGraphSetConditional(h, (counts[kActive] > wnext && it <= (unsigned long long)limit) ? 1u : 0u);
}

// set status for systems: active probes (lanczos flag) -> `on`, others -> kIdle
__global__ void k_set_status(int nsys, int ns, const int* __restrict__ probe_active, int on,
                             int* __restrict__ sysi) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nsys) return;
  const int b = s / ns;
  sysi[(long long)s * kSysI + kStatus] = (probe_active == nullptr || probe_active[b]) ? on : kIdle;
}

// change status from -> to
__global__ void k_remap_status(int nsys, int from, int to, int* __restrict__ sysi) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nsys) return;
  int* si = sysi + (long long)s * kSysI;
  if (si[kStatus] == from) si[kStatus] = to;
}

// x64 += (double) x32 for systems whose refinement counter says they were corrected
template <typename TH, typename TL>
__global__ void k_accumulate(long long nd, int nsys, const int* __restrict__ sysi, int mask,
                             int round, const cpx<TL>* __restrict__ xl, cpx<TH>* __restrict__ xh,
                             int set) {
  const int s = blockIdx.y;
  if (!((mask >> sysi[(long long)s * kSysI + kStatus]) & 1)) return;
  if (round >= 0 && sysi[(long long)s * kSysI + kRestarts] != round) return;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < nd;
       p += (long long)gridDim.x * blockDim.x) {
    const long long q = (long long)s * nd + p;
    const cpx<TL> a = xl[q];
    if (set)
      xh[q] = mk<TH>((TH)a.re, (TH)a.im);
    else
      xh[q] = mk<TH>(xh[q].re + (TH)a.re, xh[q].im + (TH)a.im);
  }
}

// density response: dens_b = 4 sum_n psi_n (.) Re x_{b,n}  (Algorithm 1, inner loop)
template <typename TX, typename TP>
__global__ void __launch_bounds__(256) k_density(long long nd, int ns, int nb,
                                                 const TP* __restrict__ psi,
                                                 const cpx<TX>* __restrict__ x,
                                                 const int* __restrict__ probe_active,
                                                 double* __restrict__ dens) {
  const int b = blockIdx.y;
  if (probe_active && !probe_active[b]) return;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < nd;
       p += (long long)gridDim.x * blockDim.x) {
    TP acc = 0;
    for (int n = 0; n < ns; ++n)
      acc += psi[(long long)n * nd + p] * (TP)x[((long long)b * ns + n) * nd + p].re;
    dens[(long long)b * nd + p] = 4.0 * (double)acc;
  }
}

// -------------------------------------------------------------------------------------------
// double-float form of the mixed form's FP64 solution (float4 per complex value:
// re.hi, re.lo, im.hi, im.lo)
// -------------------------------------------------------------------------------------------
__global__ void k_d2df(const double* __restrict__ a, float2* __restrict__ b, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double v = a[i];
    const float h = __double2float_rn(v);
    b[i] = make_float2(h, __double2float_rn(v - (double)h));
  }
}

__global__ void k_accumulate_df(long long nd, const int* __restrict__ sysi, int mask, int round,
                                const cpx<float>* __restrict__ xl, float4* __restrict__ xh,
                                int set) {
  const int s = blockIdx.y;
  if (!((mask >> sysi[(long long)s * kSysI + kStatus]) & 1)) return;
  if (round >= 0 && sysi[(long long)s * kSysI + kRestarts] != round) return;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < nd;
       p += (long long)gridDim.x * blockDim.x) {
    const long long q = (long long)s * nd + p;
    const cpx<float> a = xl[q];
    if (set) {
      xh[q] = make_float4(a.re, 0.f, a.im, 0.f);
    } else {
      const float4 v = xh[q];
      const df re = df_add(df{v.x, v.y}, df{a.re, 0.f}), im = df_add(df{v.z, v.w}, df{a.im, 0.f});
      xh[q] = make_float4(re.hi, re.lo, im.hi, im.lo);
    }
  }
}

__global__ void __launch_bounds__(256) k_density_df(long long nd, int ns, int nb,
                                                    const double* __restrict__ psi,
                                                    const float4* __restrict__ x,
                                                    const int* __restrict__ probe_active,
                                                    double* __restrict__ dens) {
  const int b = blockIdx.y;
  if (probe_active && !probe_active[b]) return;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < nd;
       p += (long long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int n = 0; n < ns; ++n) {
      const float4 v = x[((long long)b * ns + n) * nd + p];
      acc += psi[(long long)n * nd + p] * ((double)v.x + (double)v.y);
    }
    dens[(long long)b * nd + p] = 4.0 * acc;
  }
}

// cd[s][g][l] = gamma dV sum_e chi(e) x_s(idx_e) with double-float products and sums; the
// block's partial sums are combined in double-float through shared memory
__global__ void __launch_bounds__(128) k_proj_dots_df(DfAux aux, long long nd,
                                                      const float4* __restrict__ vec,
                                                      const int* __restrict__ sysi, int mask,
                                                      cpx<double>* __restrict__ cd) {
  const int g = blockIdx.x, s = blockIdx.y;
  if (sysi && !selected(sysi, s, mask)) return;
  __shared__ df sh[128 * 2 * kProjChunk];
  const float4* v = vec + (long long)s * nd;
  df acc[2 * kProjChunk];
#pragma unroll
  for (int q = 0; q < 2 * kProjChunk; ++q) acc[q] = df{0.f, 0.f};
  for (int e = aux.nl.g_off[g] + threadIdx.x; e < aux.nl.g_off[g + 1]; e += blockDim.x) {
    const float4 xv = v[aux.nl.g_idx[e]];
#pragma unroll
    for (int l = 0; l < kProjChunk; ++l) {
      const df ch{aux.nl.g_chi[(long long)e * kProjChunk + l], aux.g_chi_lo[(long long)e * kProjChunk + l]};
      acc[2 * l] = df_fma(acc[2 * l], ch, df{xv.x, xv.y});
      acc[2 * l + 1] = df_fma(acc[2 * l + 1], ch, df{xv.z, xv.w});
    }
  }
#pragma unroll
  for (int q = 0; q < 2 * kProjChunk; ++q) sh[q * 128 + threadIdx.x] = acc[q];
  __syncthreads();
  for (int w = 64; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
#pragma unroll
      for (int q = 0; q < 2 * kProjChunk; ++q)
        sh[q * 128 + threadIdx.x] = df_add(sh[q * 128 + threadIdx.x], sh[q * 128 + threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x < kProjChunk) {
    const int l = threadIdx.x;
    const df cf{aux.nl.coef[g * kProjChunk + l], aux.coef_lo[g * kProjChunk + l]};
    const df re = df_mul(cf, sh[(2 * l) * 128]), im = df_mul(cf, sh[(2 * l + 1) * 128]);
    cd[((long long)s * aux.nl.ngroup + g) * kProjChunk + l] = mk<double>(df_val(re), df_val(im));
  }
}

// -------------------------------------------------------------------------------------------
// launchers
// -------------------------------------------------------------------------------------------
template <typename T>
cudaError_t proj_dots(const NonlocalDev<T>& nl, long long nd, int nsys, const cpx<T>* vec,
                      const int* sysi, int mask, cpx<T>* cd, cudaStream_t st) {
  if (nl.ngroup == 0 || nsys == 0) return cudaSuccess;
  dim3 grid(nl.ngroup, nsys);
  k_proj_dots<T><<<grid, 128, 0, st>>>(nl, nd, vec, sysi, mask, cd);
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t apply_h(const Stencil<T>& st, const T* vloc, const NonlocalDev<T>& nl, long long nd,
                    int count, const cpx<T>* x, const cpx<T>* sigma, cpx<T>* cd, cpx<T>* y,
                    cudaStream_t s) {
  cudaError_t e = proj_dots<T>(nl, nd, count, x, nullptr, 0, cd, s);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)((nd + 255) / 256), count);
  k_apply_h<T><<<grid, 256, 0, s>>>(st, vloc, nl, nd, x, sigma, cd, y);
  note_launch();
  return cudaGetLastError();
}

cudaError_t cocg_scalars(int nsys, int tiles, const double* part, double* sysd, int* sysi,
                         int kind, int mask, double tol, double inner_tol, int maxit,
                         int max_restart, cudaStream_t s, int stride, const int* list) {
  if (nsys <= 0) return cudaSuccess;
  k_scalars<<<(nsys + 3) / 4, 128, 0, s>>>(nsys, tiles, stride > 0 ? stride : tiles, part, sysd,
                                           sysi, kind, mask, tol, inner_tol, maxit, max_restart,
                                           list);
  note_launch();
  return cudaGetLastError();
}

cudaError_t count_status(int nsys, const int* sysi, int* counts, cudaStream_t s, int* list) {
  k_count_status<<<1, 1024, 0, s>>>(nsys, sysi, counts, list);
  note_launch();
  return cudaGetLastError();
}

cudaError_t loop_cond(const int* counts, unsigned long long* ctl, cudaGraphConditionalHandle h,
                      int wnext, int limit, int add_iters, int add_launches, cudaStream_t s) {
  k_loop_cond<<<1, 1, 0, s>>>(counts, ctl, h, wnext, limit, add_iters, add_launches);
  note_launch();
  return cudaGetLastError();
}

cudaError_t set_status(int nsys, int ns, const int* probe_active, int on, int* sysi,
                       cudaStream_t s) {
  k_set_status<<<(nsys + 255) / 256, 256, 0, s>>>(nsys, ns, probe_active, on, sysi);
  note_launch();
  return cudaGetLastError();
}

cudaError_t remap_status(int nsys, int from, int to, int* sysi, cudaStream_t s) {
  k_remap_status<<<(nsys + 255) / 256, 256, 0, s>>>(nsys, from, to, sysi);
  note_launch();
  return cudaGetLastError();
}

template <typename TH, typename TL>
cudaError_t accumulate(long long nd, int nsys, const int* sysi, int mask, int round,
                       const cpx<TL>* xl, cpx<TH>* xh, int set, cudaStream_t s) {
  dim3 grid((unsigned)std::min<long long>((nd + 255) / 256, 64), nsys);
  k_accumulate<TH, TL><<<grid, 256, 0, s>>>(nd, nsys, sysi, mask, round, xl, xh, set);
  note_launch();
  return cudaGetLastError();
}

template <typename TX, typename TP>
cudaError_t density(long long nd, int ns, int nb, const TP* psi, const cpx<TX>* x,
                    const int* probe_active, double* dens, cudaStream_t s) {
  dim3 grid((unsigned)std::min<long long>((nd + 255) / 256, 256), nb);
  k_density<TX, TP><<<grid, 256, 0, s>>>(nd, ns, nb, psi, x, probe_active, dens);
  note_launch();
  return cudaGetLastError();
}

cudaError_t convert_d2df(const double* a, float2* b, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_d2df<<<(unsigned)std::min<long long>((n + 255) / 256, 4096), 256, 0, s>>>(a, b, n);
  note_launch();
  return cudaGetLastError();
}

cudaError_t accumulate_df(long long nd, int nsys, const int* sysi, int mask, int round,
                          const cpx<float>* xl, float4* xh, int set, cudaStream_t s) {
  if (nsys <= 0) return cudaSuccess;
  dim3 grid((unsigned)std::min<long long>((nd + 255) / 256, 256), nsys);
  k_accumulate_df<<<grid, 256, 0, s>>>(nd, sysi, mask, round, xl, xh, set);
  note_launch();
  return cudaGetLastError();
}

cudaError_t density_df(long long nd, int ns, int nb, const double* psi, const float4* x,
                       const int* probe_active, double* dens, cudaStream_t s) {
  dim3 grid((unsigned)std::min<long long>((nd + 255) / 256, 256), nb);
  k_density_df<<<grid, 256, 0, s>>>(nd, ns, nb, psi, x, probe_active, dens);
  note_launch();
  return cudaGetLastError();
}

cudaError_t proj_dots_df(const DfAux& aux, long long nd, int nsys, const float4* x,
                         const int* sysi, int mask, cpx<double>* cd, cudaStream_t s) {
  if (aux.nl.ngroup == 0 || nsys == 0) return cudaSuccess;
  dim3 grid(aux.nl.ngroup, nsys);
  k_proj_dots_df<<<grid, 128, 0, s>>>(aux, nd, x, sysi, mask, cd);
  note_launch();
  return cudaGetLastError();
}

// explicit instantiations
template cudaError_t proj_dots<double>(const NonlocalDev<double>&, long long, int,
                                       const cpx<double>*, const int*, int, cpx<double>*,
                                       cudaStream_t);
template cudaError_t proj_dots<float>(const NonlocalDev<float>&, long long, int,
                                      const cpx<float>*, const int*, int, cpx<float>*,
                                      cudaStream_t);
template cudaError_t apply_h<double>(const Stencil<double>&, const double*,
                                     const NonlocalDev<double>&, long long, int,
                                     const cpx<double>*, const cpx<double>*, cpx<double>*,
                                     cpx<double>*, cudaStream_t);
template cudaError_t apply_h<float>(const Stencil<float>&, const float*, const NonlocalDev<float>&,
                                    long long, int, const cpx<float>*, const cpx<float>*,
                                    cpx<float>*, cpx<float>*, cudaStream_t);
template cudaError_t accumulate<double, float>(long long, int, const int*, int, int,
                                               const cpx<float>*, cpx<double>*, int, cudaStream_t);
template cudaError_t density<double, double>(long long, int, int, const double*,
                                             const cpx<double>*, const int*, double*,
                                             cudaStream_t);
template cudaError_t density<float, float>(long long, int, int, const float*, const cpx<float>*,
                                           const int*, double*, cudaStream_t);
template cudaError_t density<double, float>(long long, int, int, const float*,
                                            const cpx<double>*, const int*, double*,
                                            cudaStream_t);

}  // namespace rpa
