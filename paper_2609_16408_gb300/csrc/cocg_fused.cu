// Fused COCG iteration for the batched Sternheimer systems (Eq. 4, Section 4).
//
// Per iteration and active system (unconjugated bilinear form a^T b):
//   K_A  p_k = r_k + beta_{k-1} p_{k-1};  w = (H - sigma) p_k;  partial mu = p_k^T w
//   S1   alpha = rho / mu
//   K_B  x += alpha p_k;  r -= alpha w;  partials ||r||^2, r^T r;  projector sums of r
//   S2   convergence test, beta = rho'/rho, projector coefficients of the next direction
// K_A is blocked in 2.5 dimensions: a block owns a 32 x 8 column tile of the grid and walks
// along z, keeping the 2R+1 values of its column in registers and the current xy plane
// (with an R-wide halo) in shared memory, so every input value is read from memory about
// once.  The direction vector is double-buffered (read p_{k-1}, write p_k) because
// neighbouring blocks read p_{k-1} in their halo.  The nonlocal term uses the projector
// coefficients of p_k, formed linearly from those of r_k and p_{k-1} by S2.
#include <cuda_runtime.h>

#include "cocg.cuh"
#include "cocg_fused.cuh"
#include "fused_dev.cuh"


namespace rpa {

constexpr int kFTX = 32, kFTY = 8;

// Direction update + H apply, 2.5-D blocked (see the file comment).  All offsets inside a
// system are 32-bit (N_d < 2^31); stencil neighbours are read from shared memory at
// compile-time offsets from a per-thread base; FIRST marks the first iteration of a solve
// (p_k = r_k, no previous direction).  The projector term of w is added by the update
// kernel (k_update_dots); this kernel applies the local part of H - sigma.
template <typename T, int R, bool FIRST>
__global__ void __launch_bounds__(kFTX * kFTY, sizeof(T) == 4 ? 3 : 2)
    k_dirmatvec(CocgView<T> cv, FusedBufs<T> fb) {
  const int s = cv.list ? cv.list[blockIdx.y] : blockIdx.y;
  if (s < 0 || cv.sysi[(long long)s * kSysI + kStatus] != kActive) return;
  constexpr int EXN = kFTX + 2 * R, EYN = kFTY + 2 * R;
  constexpr int PLN = EXN * EYN;
  constexpr int NHALO = PLN - kFTX * kFTY;
  constexpr int HPT = (NHALO + kFTX * kFTY - 1) / (kFTX * kFTY);
  __shared__ cpx<T> pl[2 * PLN];
  const Stencil<T>& st = cv.st;
  const int nx = st.nx, ny = st.ny, nz = st.nz;
  const int plane = nx * ny;
  const int ntx = (nx + kFTX - 1) / kFTX;
  const int tx0 = (blockIdx.x % ntx) * kFTX, ty0 = (blockIdx.x / ntx) * kFTY;
  const int z0 = blockIdx.z * fb.zchunk, z1 = min(z0 + fb.zchunk, nz);
  const int lx = threadIdx.x & (kFTX - 1), ly = threadIdx.x / kFTX;
  const int gx = tx0 + lx, gy = ty0 + ly;
  const bool valid = gx < nx && gy < ny;
  const long long sbase = (long long)s * cv.nd;
  const cpx<T>* __restrict__ r = cv.r + sbase;
  const cpx<T>* __restrict__ po = fb.p_in + sbase;
  cpx<T>* __restrict__ pn = fb.p_out + sbase;
  cpx<T>* __restrict__ w = cv.w + sbase;
  const T* __restrict__ vloc = cv.vloc;
  const double* sd = cv.sysd + (long long)s * kSysD;
  const cpx<T> be = mk<T>((T)sd[kBeta], (T)sd[kBeta + 1]);
  const int b = s / cv.ns, n = s - b * cv.ns;
  const cpx<T> sigma = mk<T>((T)cv.eps[n], (T)cv.omega[b]);
  // xy offsets (fixed along z) of the own column and of this thread's halo elements
  int own_xy;
  {
    const int x = wrap_or_neg(gx, nx, st.bcx), y = wrap_or_neg(gy, ny, st.bcy);
    own_xy = (x < 0 || y < 0) ? -1 : x + nx * y;
  }
  int halo_xy[HPT];
  cpx<T>* halo_s[HPT];
#pragma unroll
  for (int k = 0; k < HPT; ++k) {
    const int hi = threadIdx.x + k * kFTX * kFTY;  // index into the ring enumeration
    halo_s[k] = nullptr;
    halo_xy[k] = -1;
    if (hi < NHALO) {
      // ring: R rows above, then kFTY middle rows (left R, right R), then R rows below
      int ey, ex;
      if (hi < R * EXN) {
        ey = hi / EXN;
        ex = hi - ey * EXN;
      } else if (hi < R * EXN + kFTY * 2 * R) {
        const int t = hi - R * EXN;
        ey = R + t / (2 * R);
        const int c = t - (ey - R) * 2 * R;
        ex = (c < R) ? c : kFTX + c;
      } else {
        const int t = hi - R * EXN - kFTY * 2 * R;
        ey = R + kFTY + t / EXN;
        ex = t - (ey - R - kFTY) * EXN;
      }
      halo_s[k] = pl + ey * EXN + ex;
      const int x = wrap_or_neg(tx0 - R + ex, nx, st.bcx), y = wrap_or_neg(ty0 - R + ey, ny, st.bcy);
      halo_xy[k] = (x < 0 || y < 0) ? -1 : x + nx * y;
    }
  }
  cpx<T>* const own_s = pl + (ly + R) * EXN + (lx + R);
  auto zoff = [&](int z) -> int {
    const int zz = wrap_or_neg(z, nz, st.bcz);
    return zz < 0 ? -1 : zz * plane;
  };
  auto ld = [&](int q, cpx<T>& rv, cpx<T>& pv) {
    if (q < 0) {
      rv = mk<T>((T)0, (T)0);
      pv = rv;
    } else {
      rv = r[q];
      if (!FIRST) pv = po[q];
    }
  };
  auto comb = [&](const cpx<T>& rv, const cpx<T>& pv) -> cpx<T> {
    if (FIRST) return rv;
    return cadd(rv, cmul(be, pv));
  };
  cpx<T> zq[2 * R + 1];
#pragma unroll
  for (int i = 0; i < 2 * R; ++i) {
    const int zo = zoff(z0 - R + i);
    cpx<T> rv, pv;
    ld((zo < 0 || own_xy < 0) ? -1 : zo + own_xy, rv, pv);
    zq[i] = comb(rv, pv);
  }
  cpx<T> nq_r, nq_p, h_r[HPT], h_p[HPT];
  auto prefetch = [&](int z) {
    const int zo = zoff(z + R);
    ld((zo < 0 || own_xy < 0) ? -1 : zo + own_xy, nq_r, nq_p);
    const int zp = z * plane;
#pragma unroll
    for (int k = 0; k < HPT; ++k) ld(halo_xy[k] < 0 ? -1 : zp + halo_xy[k], h_r[k], h_p[k]);
  };
  if (z0 < z1) prefetch(z0);
  using A = dacc_t<T>;
  A acc_re = 0, acc_im = 0;
  const T c0 = st.c0;
  for (int z = z0; z < z1; ++z) {
    const int bo = ((z - z0) & 1) * PLN;
    zq[2 * R] = comb(nq_r, nq_p);
    own_s[bo] = zq[R];
#pragma unroll
    for (int k = 0; k < HPT; ++k)
      if (halo_s[k]) halo_s[k][bo] = comb(h_r[k], h_p[k]);
    if (z + 1 < z1) prefetch(z + 1);  // in flight while this plane is computed
    __syncthreads();
    if (valid) {
      const int q = own_xy + z * plane;
      const cpx<T> c = zq[R];
      const cpx<T>* cs = own_s + bo;
      const T dg = c0 + vloc[q];
      cpx<T> a = mk<T>(dg * c.re - (sigma.re * c.re - sigma.im * c.im),
                       dg * c.im - (sigma.re * c.im + sigma.im * c.re));
#pragma unroll
      for (int m = 1; m <= R; ++m) {
        a = caxpy_r(a, st.cx[m], cadd(cs[-m], cs[m]));
        a = caxpy_r(a, st.cy[m], cadd(cs[-m * EXN], cs[m * EXN]));
        a = caxpy_r(a, st.cz[m], cadd(zq[R - m], zq[R + m]));
      }
      w[q] = a;
      pn[q] = c;
      acc_re += (A)c.re * a.re - (A)c.im * a.im;
      acc_im += (A)c.re * a.im + (A)c.im * a.re;
    }
#pragma unroll
    for (int i = 0; i < 2 * R; ++i) zq[i] = zq[i + 1];
  }
  A acc2[2] = {acc_re, acc_im};
  __shared__ A sha[8 * 2];
  block_sum_t<A, 2>(acc2, sha);
  if (threadIdx.x == 0) {
    const int pid = blockIdx.x + gridDim.x * blockIdx.z;
    double* pp = cv.part + ((long long)s * cv.tiles + pid) * 4;
    pp[0] = (double)acc2[0];
    pp[1] = (double)acc2[1];
  }
}

// x += alpha p, r -= alpha w; partials ||r||^2 (slot 0) and r^T r (slots 2, 3).  The
// updated r of the tile is kept in shared memory; then each warp takes whole projector
// groups touching the tile (their entries are sorted by grid index, so a group's entries in
// this tile are one contiguous range), reduces coef * chi * r over the range with shuffles
// and adds the tile's contribution to cr[s][g][l] with one atomic per value.
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 5 : 1) k_update_dots(CocgView<T> cv, FusedBufs<T> fb) {
  const int s = cv.list ? cv.list[blockIdx.y] : blockIdx.y;
  if (s < 0 || cv.sysi[(long long)s * kSysI + kStatus] != kActive) return;
  __shared__ double sh[8 * 3];
  __shared__ cpx<T> sr[kTile];
  __shared__ cpx<T> swn[kTile];  // projector term V_nl p of the tile's points
  const long long nd = cv.nd;
  const double* sd = cv.sysd + (long long)s * kSysD;
  const cpx<T> al = mk<T>((T)sd[kAlpha], (T)sd[kAlpha + 1]);
  const bool nl = cv.nl.ngroup > 0;
  using A = dacc_t<T>;
  A a0 = 0, a1 = 0, a2 = 0;
  const long long t0 = (long long)blockIdx.x * kTile;
  const long long t1 = min(t0 + kTile, nd);
  const cpx<T>* __restrict__ pp_ = fb.p_out + (long long)s * nd;
  const cpx<T>* __restrict__ ww_ = cv.w + (long long)s * nd;
  cpx<T>* __restrict__ xx_ = cv.x + (long long)s * nd;
  cpx<T>* __restrict__ rr_ = cv.r + (long long)s * nd;
  constexpr int U = kTile / 256;  // points per thread, all loads issued before any store
  cpx<T> pv[U], wv[U], xv[U], rv0[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const long long p = t0 + threadIdx.x + u * 256;
    if (p < t1) {
      pv[u] = pp_[p];
      wv[u] = ww_[p];
      xv[u] = xx_[p];
      rv0[u] = rr_[p];
    }
  }
  // w holds the local part (H_loc - sigma) p only.  Without projectors r_{k+1} = r - alpha w
  // is final at once.  With them one pass over the tile's projector entries, whole warps per
  // projector group (entries of a group in the tile are one contiguous range of distinct
  // points), both adds chi * cp (the projector term V_nl p) to the tile's points in shared
  // memory and forms the sums chi^T rhat of rhat = r - alpha w_loc, reduced with shuffles
  // and added to cr[s][g][l] with one atomic per value; r_{k+1} = rhat - alpha V_nl p follows
  // after the pass, and the part alpha chi^T V_nl p = alpha S cp of the sums is taken off
  // per system afterwards (k_proj_next).
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const long long p = t0 + threadIdx.x + u * 256;
    if (p < t1) {
      xx_[p] = cadd(xv[u], cmul(al, pv[u]));
      const cpx<T> rv = csub(rv0[u], cmul(al, wv[u]));
      if (nl) {
        sr[p - t0] = rv;
        swn[p - t0] = mk<T>((T)0, (T)0);
      } else {
        rr_[p] = rv;
        a0 += (A)rv.re * rv.re + (A)rv.im * rv.im;
        a1 += (A)rv.re * rv.re - (A)rv.im * rv.im;
        a2 += (A)2 * rv.re * rv.im;
      }
    }
  }
  if (nl) {
    __syncthreads();
    cpx<T>* cr = fb.cr + (long long)s * cv.nl.ngroup * kProjChunk;
    const cpx<T>* cpg = fb.cp + (long long)s * cv.nl.ngroup * kProjChunk;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q0 = fb.tile_roff[blockIdx.x], q1 = fb.tile_roff[blockIdx.x + 1];
    for (int q = q0 + warp; q < q1; q += (int)(blockDim.x >> 5)) {
      const int g = fb.tile_ranges[3 * q], e0 = fb.tile_ranges[3 * q + 1],
                e1 = fb.tile_ranges[3 * q + 2];
      cpx<T> cg[kProjChunk];
#pragma unroll
      for (int l = 0; l < kProjChunk; ++l) cg[l] = cpg[g * kProjChunk + l];
      T a[2 * kProjChunk];
#pragma unroll
      for (int i = 0; i < 2 * kProjChunk; ++i) a[i] = (T)0;
      // entries of the range, one per lane, the next one fetched while this one is used
      int e = e0 + lane;
      int ix = e < e1 ? cv.nl.g_idx[e] : 0;
      T ch[kProjChunk] = {0, 0, 0, 0};
      if (e < e1) load_chi4(cv.nl.g_chi + (long long)e * kProjChunk, ch);
      while (e < e1) {
        const int en = e + 32;
        int ixn = 0;
        T chn[kProjChunk] = {0, 0, 0, 0};
        if (en < e1) {
          ixn = cv.nl.g_idx[en];
          load_chi4(cv.nl.g_chi + (long long)en * kProjChunk, chn);
        }
        const cpx<T> rv = sr[ix - t0];
        cpx<T> v = mk<T>((T)0, (T)0);
#pragma unroll
        for (int l = 0; l < kProjChunk; ++l) {
          a[2 * l] += ch[l] * rv.re;
          a[2 * l + 1] += ch[l] * rv.im;
          v = caxpy_r(v, ch[l], cg[l]);
          ch[l] = chn[l];
        }
        atomicAdd(&swn[ix - t0].re, v.re);
        atomicAdd(&swn[ix - t0].im, v.im);
        ix = ixn;
        e = en;
      }
      // butterfly reduction: every lane ends with the full sums
#pragma unroll
      for (int i = 0; i < 2 * kProjChunk; ++i)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a[i] += __shfl_xor_sync(0xffffffffu, a[i], o);
      if (lane < kProjChunk) {
        T re = a[0], im = a[1];
#pragma unroll
        for (int l = 1; l < kProjChunk; ++l)
          if (lane == l) {
            re = a[2 * l];
            im = a[2 * l + 1];
          }
        const T cf = cv.nl.coef[g * kProjChunk + lane];
        atomicAdd(&cr[g * kProjChunk + lane].re, cf * re);
        atomicAdd(&cr[g * kProjChunk + lane].im, cf * im);
      }
    }
    __syncthreads();
    for (long long p = t0 + threadIdx.x; p < t1; p += blockDim.x) {
      const cpx<T> rv = csub(sr[p - t0], cmul(al, swn[p - t0]));
      rr_[p] = rv;
      a0 += (A)rv.re * rv.re + (A)rv.im * rv.im;
      a1 += (A)rv.re * rv.re - (A)rv.im * rv.im;
      a2 += (A)2 * rv.re * rv.im;
    }
  }
  A acc[3] = {a0, a1, a2};
  block_sum_t<A, 3>(acc, reinterpret_cast<A*>(sh));
  if (threadIdx.x == 0) {
    double* pp = cv.part + ((long long)s * cv.tiles + blockIdx.x) * 4;
    pp[0] = (double)acc[0];
    pp[2] = (double)acc[1];
    pp[3] = (double)acc[2];
  }
}

// S2 with the projector bookkeeping.  After the scalar step (kind 2), every still-active
// system forms cp = cr + beta cp and clears cr.  One block per system.  With corr, cr holds
// the sums chi^T rhat of the update kernel (rhat = r - alpha w_loc): the projector part
// alpha chi^T V_nl p = alpha S cp is taken off first, S the projector overlap blocks, with
// the system's cp (still that of the last direction) staged in shared memory.  Then
// p^T V_nl p = sum over projectors of cp^2 / (gamma dV) (cp = gamma dV chi^T p; unconjugated
// square) goes to sysd[kNlDot] for the next alpha step.
constexpr int kProjNextThreads = 128;
template <typename T>
__global__ void __launch_bounds__(kProjNextThreads)
    k_proj_next(int nsys, NonlocalDev<T> nl, double* __restrict__ sysd,
                const int* __restrict__ sysi, int init, cpx<T>* __restrict__ cp,
                cpx<T>* __restrict__ cr, const int* __restrict__ list, int corr, int stage) {
  const int i = blockIdx.x;
  if (i >= nsys) return;
  const int s = list ? list[i] : i;
  if (s < 0 || sysi[(long long)s * kSysI + kStatus] != kActive) return;
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  // ngroup x 4 coefficients of the system (corr; read in place when they exceed 48 KB)
  cpx<T>* scp = reinterpret_cast<cpx<T>*>(dyn_smem);
  const int ngroup = nl.ngroup, nv = ngroup * kProjChunk;
  double* sd = sysd + (long long)s * kSysD;
  const cpx<T> be = init ? mk<T>((T)0, (T)0) : mk<T>((T)sd[kBeta], (T)sd[kBeta + 1]);
  cpx<T>* p = cp + (long long)s * nv;
  cpx<T>* q = cr + (long long)s * nv;
  if (corr) {
    if (stage) {
      for (int j = threadIdx.x; j < nv; j += blockDim.x) scp[j] = p[j];
      __syncthreads();
    } else {
      scp = p;
    }
    const cpx<T> al = mk<T>((T)sd[kAlpha], (T)sd[kAlpha + 1]);
    for (int j = threadIdx.x; j < nv; j += blockDim.x) {
      const int g = j / kProjChunk, l = j - g * kProjChunk;
      cpx<T> v = mk<T>((T)0, (T)0);
      const int k0 = nl.s_off[g], k1 = nl.s_off[g + 1];
#pragma unroll 4
      for (int k = k0; k < k1; ++k) {
        const T* blk = nl.s_blk + (long long)k * 16 + l * 4;
        const cpx<T>* ph = scp + nl.s_nbr[k] * kProjChunk;
#pragma unroll
        for (int m = 0; m < kProjChunk; ++m) v = caxpy_r(v, blk[m], ph[m]);
      }
      q[j] = csub(q[j], cmul(al, mk<T>(nl.coef[j] * v.re, nl.coef[j] * v.im)));
    }
    if (!stage) __syncthreads();  // every read of the old coefficients in place is done
  }
  double dre = 0.0, dim = 0.0;
  for (int j = threadIdx.x; j < nv; j += blockDim.x) {
    const cpx<T> v = init ? q[j] : cadd(q[j], cmul(be, p[j]));
    p[j] = v;
    q[j] = mk<T>((T)0, (T)0);
    const double cf = (double)nl.coef[j];
    if (cf != 0.0) {
      const double a = (double)v.re, b = (double)v.im;
      dre += (a * a - b * b) / cf;
      dim += 2.0 * a * b / cf;
    }
  }
  double acc[2] = {dre, dim};
  __shared__ double shd[(kProjNextThreads / 32) * 2];
  block_sum_t<double, 2>(acc, shd);
  if (threadIdx.x == 0) {
    sd[kNlDot] = acc[0];
    sd[kNlDot + 1] = acc[1];
  }
}

template <typename T>
static void launch_proj_next(const CocgView<T>& cv, const FusedBufs<T>& fb, int nsys,
                             const int* list, int init, int corr, cudaStream_t s) {
  size_t smem = corr ? sizeof(cpx<T>) * cv.nl.ngroup * kProjChunk : 0;
  const int stage = smem > 0 && smem <= 48 * 1024;
  if (!stage) smem = 0;
  k_proj_next<T><<<nsys, kProjNextThreads, smem, s>>>(nsys, cv.nl, cv.sysd, cv.sysi, init,
                                                      fb.cp, fb.cr, list, corr, stage);
}

// -------------------------------------------------------------------------------------------
template <typename T, int R>
static void launch_dirmatvec(const CocgView<T>& cv, const FusedBufs<T>& fb, cudaStream_t s) {
  dim3 grid(fb.ntiles_xy, fb.nact, fb.nzchunk);
  if (fb.first)
    k_dirmatvec<T, R, true><<<grid, kFTX * kFTY, 0, s>>>(cv, fb);
  else
    k_dirmatvec<T, R, false><<<grid, kFTX * kFTY, 0, s>>>(cv, fb);
}

template <typename T>
cudaError_t launch_dirmatvec_only(const CocgView<T>& cv, const FusedBufs<T>& fb, cudaStream_t s) {
  if (is_band(fb.row_ty)) {
    if constexpr (sizeof(T) == 4) {
      cudaError_t e = launch_dirmatvec_band(cv, fb, s);
      note_launch();
      return e;
    } else {
      return cudaErrorInvalidValue;  // FP32 only
    }
  }
  if (fb.row_ty == kTileX2Packed) {
    if constexpr (sizeof(T) == 4) {
      cudaError_t e = launch_dirmatvec_x2p(cv, fb, s);
      note_launch();
      return e;
    } else {
      return cudaErrorInvalidValue;  // FP32 only
    }
  }
  if (is_x2(fb.row_ty)) {
    if constexpr (sizeof(T) == 4) {
      cudaError_t e = launch_dirmatvec_x2(cv, fb, s);
      note_launch();
      return e;
    } else {
      return cudaErrorInvalidValue;  // FP32 only
    }
  }
  if (fb.row_ty > 0) {
    cudaError_t e = launch_dirmatvec_rows<T>(cv, fb, s);
    note_launch();
    return e;
  }
  switch (cv.st.R) {
    case 1: launch_dirmatvec<T, 1>(cv, fb, s); break;
    case 2: launch_dirmatvec<T, 2>(cv, fb, s); break;
    case 3: launch_dirmatvec<T, 3>(cv, fb, s); break;
    case 4: launch_dirmatvec<T, 4>(cv, fb, s); break;
    case 5: launch_dirmatvec<T, 5>(cv, fb, s); break;
    case 6: launch_dirmatvec<T, 6>(cv, fb, s); break;
    case 7: launch_dirmatvec<T, 7>(cv, fb, s); break;
    default: launch_dirmatvec<T, 8>(cv, fb, s); break;
  }
  note_launch();
  return cudaGetLastError();
}
template cudaError_t launch_dirmatvec_only<float>(const CocgView<float>&, const FusedBufs<float>&,
                                                  cudaStream_t);
template cudaError_t launch_dirmatvec_only<double>(const CocgView<double>&,
                                                   const FusedBufs<double>&, cudaStream_t);

template <typename T>
cudaError_t fused_iteration(const CocgView<T>& cv, const FusedBufs<T>& fb, double tol, int maxit,
                            cudaStream_t s, cudaEvent_t* ev) {
  if (ev) cudaEventRecord(ev[0], s);
  if (ev) cudaEventRecord(ev[1], s);
  {
    cudaError_t e0 = launch_dirmatvec_only<T>(cv, fb, s);
    if (e0 != cudaSuccess) return e0;
  }
  if (ev) cudaEventRecord(ev[2], s);
  cudaError_t e = cocg_scalars(fb.nact, fb.ntiles_xy * fb.nzchunk, cv.part, cv.sysd, cv.sysi, 1,
                               1 << kActive, tol, 0.0, maxit, 0, s, cv.tiles, cv.list);
  if (e != cudaSuccess) return e;
  if (ev) cudaEventRecord(ev[3], s);
  dim3 g2(fb.tiles1d, fb.nact);
  k_update_dots<T><<<g2, 256, 0, s>>>(cv, fb);
  if (ev) cudaEventRecord(ev[4], s);
  e = cocg_scalars(fb.nact, fb.tiles1d, cv.part, cv.sysd, cv.sysi, 2, 1 << kActive, tol, 0.0,
                   maxit, 0, s, cv.tiles, cv.list);
  if (e != cudaSuccess) return e;
  if (cv.nl.ngroup > 0) {
    launch_proj_next<T>(cv, fb, fb.nact, cv.list, 0, 1, s);
    note_launch();
  }
  if (ev) cudaEventRecord(ev[5], s);
  if (ev) cudaEventRecord(ev[6], s);
  note_launch(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t fused_prepare(const CocgView<T>& cv, const FusedBufs<T>& fb, cudaStream_t s,
                          int init) {
  if (cv.nl.ngroup == 0) return cudaSuccess;
  launch_proj_next<T>(cv, fb, cv.nsys, nullptr, init, 0, s);
  note_launch();
  return cudaGetLastError();
}

template cudaError_t fused_iteration<double>(const CocgView<double>&, const FusedBufs<double>&,
                                             double, int, cudaStream_t, cudaEvent_t*);
template cudaError_t fused_iteration<float>(const CocgView<float>&, const FusedBufs<float>&,
                                            double, int, cudaStream_t, cudaEvent_t*);
template cudaError_t fused_prepare<double>(const CocgView<double>&, const FusedBufs<double>&,
                                           cudaStream_t, int);
template cudaError_t fused_prepare<float>(const CocgView<float>&, const FusedBufs<float>&,
                                          cudaStream_t, int);

}  // namespace rpa
