// C ABI and host orchestration of the GB300 RPA library.
//
// Work is organised in waves of B probe-points (coarse point j, frequency w).  For every
// Lanczos step of a wave: u = nu^{1/2} q_k (mode products), Galerkin guess over the occupied
// space, B x N_s Sternheimer solves by batched COCG, density r = 4 sum_n psi_n Re(dpsi_n),
// v = nu^{1/2} r, then the Lanczos recurrence with full reorthogonalisation.  Probes leave the
// wave individually (early exit, breakdown); their systems are idle from then on.  After the
// wave, [f(T)]_{11} gives d_j (Algorithm 1).  Interpolation and the E_c sum follow per
// frequency (Section 3.2).
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "checkpoint.cuh"
#include "cocg.cuh"
#include "cocg_fused.cuh"
#include "small.cuh"

using namespace rpa;

namespace rpa {
static std::atomic<long long> g_launches{0};
void note_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

DevBuf::~DevBuf() { release(); }
cudaError_t DevBuf::ensure(size_t nbytes) {
  if (nbytes == 0) nbytes = 16;
  if (p && bytes >= nbytes) return cudaSuccess;
  release();
  cudaError_t e = cudaMalloc(&p, nbytes);
  if (e != cudaSuccess) {
    p = nullptr;
    bytes = 0;
    return e;
  }
  bytes = nbytes;
  return cudaSuccess;
}
void DevBuf::release() {
  if (p) cudaFree(p);
  p = nullptr;
  bytes = 0;
}
}  // namespace rpa

// ---------------------------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------------------------
template <typename T>
struct OpData {
  DevBuf vloc, psi, g_chi, coef, p_chi, s_blk, nuV[3], nuVt[3], nuScale;
  Stencil<T> st;
};

struct rpa_ctx {
  rpa_grid grid;
  long long nd = 0;
  double dV = 0.0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0;
  rpa_options opt;
  bool have_vloc = false, have_occ = false, have_freq = false;
  int ns = 0, nw = 0;
  std::vector<double> omega, weight;
  DevBuf eps_d, omega_d, weight_d;
  OpData<double> d64;
  OpData<float> d32;
  int ngroup = 0;
  DevBuf g_off, g_idx, p_off, p_grp, s_off, s_nbr;
  DevBuf tile_roff, tile_ranges;  // per 1-D COCG tile: (group, entry range) lists
  DevBuf lam[3];
  // interpolation operators (transposed, coarse x fine) per axis
  DevBuf interpWt[3], cnodes_d[3];
  std::vector<long long> cnodes[3];
  int interp_built = -1, stride_built[3] = {0, 0, 0};
  // wave workspace
  DevBuf Q, u64, v64, dens64, t64a, t64b, u32, t32a, t32b;
  DevBuf x, r, p, p2, w, x64, cdot, cpb, crb, part, sysd, sysi, gpart, cmat;
  // double-float (hi, lo) copies for the mixed form's refinement residual: V_loc, psi, the
  // lo parts of the projector data, and u of the current wave
  DevBuf vloc2, psi2, g_chi_lo, p_chi_lo, coef_lo, u2;
  // block Lanczos (options.lanczos_block > 1)
  DevBuf bD, bpart, bA, bB, bR, bRinv, bT, bW, blam, bsteps, bm, bfirst, bsize, bstart, bsz;
  DevBuf probe_d, pomega_d, active_d, steps_d, alpha_d, beta_d, lstate_d, coef_d, dots_d,
      dotpart_d, flags_d, dout_d, counts_d, list_d;
  int ws_nb = 0;
  int* pinned = nullptr;  // counts from the device
  std::string err;
  cudaEvent_t ev[8];
  bool have_events = false;
  // COCG kernel profiling (options.profile): events for one chunk of iterations
  cudaEvent_t pev[4 * 7];
  bool have_pev = false;
  rpa_stats* prof_stats = nullptr;
  // autotuned H-apply tiling per COCG precision (FP32, FP64) for launches over many
  // systems (bulk) and over few (tail); -1 = not tuned yet
  int tuned_ty[2][2] = {{-1, -1}, {-1, -1}};
  int nsm = 0;  // multiprocessors of the device
  // CUDA graphs of one chunk of fused COCG iterations, keyed by every launch parameter
  struct ChunkGraph {
    std::vector<unsigned char> key;
    cudaGraphExec_t exec = nullptr;
    int launches = 0;
  };
  std::vector<ChunkGraph> graphs;
  // COCG loops captured whole (options.graphs = 2): iteration and launch counters of the
  // running loop, and the loops run so far (profiling samples every kProfLoopEvery-th)
  DevBuf loopctl_d;
  long long loop_no = 0;
  int prof_cpx_bytes = 0;
  // non-fatal outcome of the current call (results are still written): RPA_ENOCONV or
  // RPA_EBREAKDOWN (the more severe is kept), with its reason
  rpa_status soft = RPA_OK;
  std::string soft_msg;
  // probe-point lanes (options.lanes > 1): helper contexts with their own stream and
  // workspace, set up from this context's inputs on first use and dropped when an input
  // changes; the projector inputs are kept on the host for them
  std::vector<rpa_ctx*> lanes;
  int hp_ng = 0;
  std::vector<int> hp_nnz, hp_nproj, hp_idx;
  std::vector<double> hp_chi, hp_gamma;
  double mem_share = 1.0;  // share of the free device memory a wave may take
  std::vector<double> eps_h;  // occupied eigenvalues (host copy)
  std::string ckpt_path;      // rpa_set_checkpoint: checkpoint file of rpa_energy_density
};

namespace rpa {
// record a non-fatal outcome of the current call (EBREAKDOWN outranks ENOCONV)
static void note_soft(rpa_ctx* c, rpa_status st, const char* msg) {
  if (c->soft == RPA_OK || (st == RPA_EBREAKDOWN && c->soft == RPA_ENOCONV)) {
    c->soft = st;
    c->soft_msg = msg;
  }
}
// the call's result: OK, or its recorded non-fatal status with the reason in last_error
static rpa_status soft_status(rpa_ctx* c) {
  const rpa_status st = c->soft;
  if (st == RPA_OK) return RPA_OK;
  c->soft = RPA_OK;
  return fail(c, st, c->soft_msg);
}
rpa_status fail(rpa_ctx* c, rpa_status st, const std::string& msg) {
  if (c) c->err = msg;
  return st;
}
rpa_status cuda_fail(rpa_ctx* c, cudaError_t e, const char* where) {
  if (c) c->err = std::string("CUDA error ") + cudaGetErrorString(e) + " in " + where;
  return RPA_ECUDA;
}
}  // namespace rpa

#define CK(call)                                                  \
  do {                                                            \
    cudaError_t e__ = (call);                                     \
    if (e__ != cudaSuccess) return rpa::cuda_fail(c, e__, #call); \
  } while (0)
#define CKS(call)                      \
  do {                                 \
    rpa_status s__ = (call);           \
    if (s__ != RPA_OK) return s__;     \
  } while (0)

// Central second-derivative weights of radius R (order 2R):
// c_m = (2/m^2) (-1)^{m+1} prod_{i=1}^{m} (R - i + 1)/(R + i), c_0 = -2 sum c_m.
static void fd_weights(int R, double* c) {
  double s = 0.0;
  for (int m = 1; m <= R; ++m) {
    double prod = 1.0;
    for (int i = 1; i <= m; ++i) prod *= (double)(R - i + 1) / (double)(R + i);
    const double v = 2.0 / ((double)m * m) * prod;
    c[m] = (m & 1) ? v : -v;
    s += c[m];
  }
  c[0] = -2.0 * s;
}

template <typename T>
static void make_stencil(const rpa_grid& g, Stencil<T>& st) {
  double c[kMaxRadius + 1];
  fd_weights(g.fd_radius, c);
  st.nx = g.n[0];
  st.ny = g.n[1];
  st.nz = g.n[2];
  st.R = g.fd_radius;
  st.bcx = g.bc[0];
  st.bcy = g.bc[1];
  st.bcz = g.bc[2];
  const double ix2 = 1.0 / (g.h[0] * g.h[0]), iy2 = 1.0 / (g.h[1] * g.h[1]),
               iz2 = 1.0 / (g.h[2] * g.h[2]);
  for (int m = 0; m <= kMaxRadius; ++m) {
    st.cx[m] = st.cy[m] = st.cz[m] = (T)0;
  }
  for (int m = 1; m <= g.fd_radius; ++m) {
    st.cx[m] = (T)(-0.5 * c[m] * ix2);
    st.cy[m] = (T)(-0.5 * c[m] * iy2);
    st.cz[m] = (T)(-0.5 * c[m] * iz2);
  }
  st.c0 = (T)(-0.5 * c[0] * (ix2 + iy2 + iz2));
}

template <typename T>
static OpData<T>& opd(rpa_ctx* c);
template <>
OpData<double>& opd<double>(rpa_ctx* c) { return c->d64; }
template <>
OpData<float>& opd<float>(rpa_ctx* c) { return c->d32; }

template <typename T>
static NonlocalDev<T> nlview(rpa_ctx* c) {
  NonlocalDev<T> nl;
  OpData<T>& o = opd<T>(c);
  nl.ngroup = c->ngroup;
  nl.g_off = c->g_off.as<int>();
  nl.g_idx = c->g_idx.as<int>();
  nl.g_chi = o.g_chi.template as<T>();
  nl.coef = o.coef.template as<T>();
  nl.p_off = c->p_off.as<int>();
  nl.p_grp = c->p_grp.as<int>();
  nl.p_chi = o.p_chi.template as<T>();
  nl.s_off = c->s_off.as<int>();
  nl.s_nbr = c->s_nbr.as<int>();
  nl.s_blk = o.s_blk.template as<T>();
  return nl;
}

static rpa_status copy_in(rpa_ctx* c, void* dst, const void* src, size_t bytes, int where) {
  CK(cudaMemcpyAsync(dst, src, bytes,
                     where == RPA_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                     c->stream));
  return RPA_OK;
}
static rpa_status copy_out(rpa_ctx* c, void* dst, const void* src, size_t bytes, int where) {
  CK(cudaMemcpyAsync(dst, src, bytes,
                     where == RPA_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     c->stream));
  return RPA_OK;
}

// ---------------------------------------------------------------------------------------------
// nu^{1/2}: eigenbases of the 1-D Laplacians (device Jacobi), then u = V S V^T q
// ---------------------------------------------------------------------------------------------
static rpa_status build_nu(rpa_ctx* c) {
  double cw[kMaxRadius + 1];
  fd_weights(c->grid.fd_radius, cw);
  double lmax = 0.0;
  for (int a = 0; a < 3; ++a) {
    const int n = c->grid.n[a];
    const double h2 = c->grid.h[a] * c->grid.h[a];
    std::vector<double> L((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) {
      L[(size_t)i * n + i] += cw[0] / h2;
      for (int m = 1; m <= c->grid.fd_radius; ++m)
        for (int sg = -1; sg <= 1; sg += 2) {
          int j = i + sg * m;
          if (c->grid.bc[a] == RPA_PERIODIC) {
            j %= n;
            if (j < 0) j += n;
          } else if (j < 0 || j >= n) {
            continue;
          }
          L[(size_t)i * n + j] += cw[m] / h2;
        }
    }
    // Gershgorin bound of |lambda| for the null-space threshold
    double rowmax = 0.0;
    for (int i = 0; i < n; ++i) {
      double rs = 0.0;
      for (int j = 0; j < n; ++j) rs += std::fabs(L[(size_t)i * n + j]);
      rowmax = std::max(rowmax, rs);
    }
    lmax += rowmax;
    DevBuf A;
    CK(A.ensure(sizeof(double) * n * n));
    CK(c->d64.nuV[a].ensure(sizeof(double) * n * n));
    CK(c->d64.nuVt[a].ensure(sizeof(double) * n * n));
    CK(c->d32.nuV[a].ensure(sizeof(float) * n * n));
    CK(c->d32.nuVt[a].ensure(sizeof(float) * n * n));
    CK(c->lam[a].ensure(sizeof(double) * n));
    CK(cudaMemcpyAsync(A.p, L.data(), sizeof(double) * n * n, cudaMemcpyHostToDevice, c->stream));
    CK(jacobi_eig(A.as<double>(), c->d64.nuV[a].as<double>(), c->lam[a].as<double>(), n,
                  c->stream));
    // transpose and FP32 copies (small: via the host)
    CK(cudaStreamSynchronize(c->stream));
    std::vector<double> V((size_t)n * n), Vt((size_t)n * n);
    CK(cudaMemcpy(V.data(), c->d64.nuV[a].p, sizeof(double) * n * n, cudaMemcpyDeviceToHost));
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) Vt[(size_t)j * n + i] = V[(size_t)i * n + j];
    std::vector<float> Vf(V.begin(), V.end()), Vtf(Vt.begin(), Vt.end());
    CK(cudaMemcpy(c->d64.nuVt[a].p, Vt.data(), sizeof(double) * n * n, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->d32.nuV[a].p, Vf.data(), sizeof(float) * n * n, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->d32.nuVt[a].p, Vtf.data(), sizeof(float) * n * n, cudaMemcpyHostToDevice));
  }
  CK(c->d64.nuScale.ensure(sizeof(double) * c->nd));
  CK(c->d32.nuScale.ensure(sizeof(float) * c->nd));
  CK(nu_scale(c->lam[0].as<double>(), c->lam[1].as<double>(), c->lam[2].as<double>(),
              c->grid.n[0], c->grid.n[1], c->grid.n[2], lmax, c->d64.nuScale.as<double>(),
              c->d32.nuScale.as<float>(), c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return RPA_OK;
}

// out_b = nu^{1/2} in_b for nb vectors (input batch stride in_bs, output contiguous).
template <typename T, typename TI, typename TO>
static rpa_status nu_half(rpa_ctx* c, const TI* in, long long in_bs, TO* out, int nb, T* ta,
                          T* tb) {
  OpData<T>& o = opd<T>(c);
  const int* n = c->grid.n;
  const long long nd = c->nd;
  int dims[3] = {n[0], n[1], n[2]};
  // forward: V^T along x, y, z, then the spectral scale
  CK((mode_product<TI, T, T>(in, in_bs, ta, nd, o.nuV[0].template as<T>(), 0, dims, n[0], nb,
                             nullptr, c->stream)));
  CK((mode_product<T, T, T>(ta, nd, tb, nd, o.nuV[1].template as<T>(), 1, dims, n[1], nb, nullptr,
                            c->stream)));
  CK((mode_product<T, T, T>(tb, nd, ta, nd, o.nuV[2].template as<T>(), 2, dims, n[2], nb,
                            o.nuScale.template as<T>(), c->stream)));
  // inverse: V along x, y, z
  CK((mode_product<T, T, T>(ta, nd, tb, nd, o.nuVt[0].template as<T>(), 0, dims, n[0], nb,
                            nullptr, c->stream)));
  CK((mode_product<T, T, T>(tb, nd, ta, nd, o.nuVt[1].template as<T>(), 1, dims, n[1], nb,
                            nullptr, c->stream)));
  CK((mode_product<T, TO, T>(ta, nd, out, nd, o.nuVt[2].template as<T>(), 2, dims, n[2], nb,
                             nullptr, c->stream)));
  return RPA_OK;
}

// ---------------------------------------------------------------------------------------------
// workspace
// ---------------------------------------------------------------------------------------------
static size_t cpx_bytes(const rpa_ctx* c) {
  return c->opt.precision == RPA_FP64 ? sizeof(cpx<double>) : sizeof(cpx<float>);
}

static long long tiles_of(long long nd) { return (nd + kTile - 1) / kTile; }
constexpr int kChunkItersMax = 4;  // COCG iterations per host check (see cocg_loop)

// 2.5-D tiling of the fused H apply: 32 x 8 column tiles, z split in chunks of <= 64 planes
static int fused_zchunk(const rpa_ctx* c) { return c->grid.n[2] <= 64 ? c->grid.n[2] : 32; }
static int fused_nzchunk(const rpa_ctx* c) {
  return (c->grid.n[2] + fused_zchunk(c) - 1) / fused_zchunk(c);
}
static int fused_ntiles_xy(const rpa_ctx* c) {
  return ((c->grid.n[0] + 31) / 32) * ((c->grid.n[1] + 7) / 8);
}
// small launches split z further (up to 8 chunks per base chunk) to fill the GPU
constexpr int kMaxZSplit = 8;
static int part_stride(const rpa_ctx* c) {
  // row tiles number at most ny per z chunk
  const long long nzc = std::min<long long>(c->grid.n[2], (long long)kMaxZSplit * fused_nzchunk(c));
  const long long fused = (long long)std::max(fused_ntiles_xy(c), c->grid.n[1]) * nzc;
  return (int)std::max<long long>(tiles_of(c->nd), fused);
}

static int gram_chunks(long long nd) {
  return (int)std::max<long long>(1, std::min<long long>(256, (nd + 4095) / 4096));
}

static size_t per_probe_bytes(const rpa_ctx* c) {
  const long long nd = c->nd, ns = c->ns;
  size_t b = (size_t)ns * nd * cpx_bytes(c) * 4;
  if (c->opt.precision != RPA_FP64 && c->opt.refine > 0)
    b += (size_t)ns * nd * sizeof(float4) + (size_t)nd * sizeof(float2);
  b += (size_t)(c->opt.lanczos_max + 1) * nd * 8 + (size_t)nd * 8 * 5 + (size_t)nd * 4 * 3;
  b += (size_t)ns * part_stride(c) * 4 * 8 + (size_t)ns * (kSysD * 8 + kSysI * 4);
  b += (size_t)ns * ns * (gram_chunks(nd) * 8 + 16);
  b += (size_t)ns * std::max(1, c->ngroup) * kProjChunk * 16 * 3;
  return b;
}

static int choose_batch(rpa_ctx* c, long long count) {
  int nb = c->opt.batch;
  if (nb <= 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) fr = (size_t)8 << 30;
    const size_t avail = (size_t)(0.55 * c->mem_share * (double)fr);
    nb = (int)std::max<size_t>(1, avail / std::max<size_t>(1, per_probe_bytes(c)));
    nb = std::min(nb, 512);
  }
  nb = std::min<long long>(nb, std::max<long long>(1, count));
  nb = std::min(nb, std::max(1, 65535 / std::max(1, c->ns)));
  return nb;
}

static rpa_status ensure_workspace(rpa_ctx* c, int nb) {
  const long long nd = c->nd, S = (long long)nb * c->ns;
  const int nl = c->opt.lanczos_max;
  const size_t cb = cpx_bytes(c);
  CK(c->Q.ensure(sizeof(double) * nb * (nl + 1) * nd));
  CK(c->u64.ensure(sizeof(double) * nb * nd));
  CK(c->v64.ensure(sizeof(double) * nb * nd));
  CK(c->dens64.ensure(sizeof(double) * nb * nd));
  CK(c->t64a.ensure(sizeof(double) * nb * nd));
  CK(c->t64b.ensure(sizeof(double) * nb * nd));
  if (c->opt.precision != RPA_FP64) {
    CK(c->u32.ensure(sizeof(float) * nb * nd));
    CK(c->t32a.ensure(sizeof(float) * nb * nd));
    CK(c->t32b.ensure(sizeof(float) * nb * nd));
    if (c->opt.refine > 0) {
      CK(c->x64.ensure(sizeof(float4) * S * nd));  // double-float pairs
      CK(c->u2.ensure(sizeof(float2) * nb * nd));
    }
  }
  CK(c->x.ensure(cb * S * nd));
  CK(c->r.ensure(cb * S * nd));
  CK(c->p.ensure(cb * S * nd));
  CK(c->p2.ensure(cb * S * nd));
  CK(c->w.ensure(cb * S * nd));
  CK(c->cdot.ensure(sizeof(cpx<double>) * S * std::max(1, c->ngroup) * kProjChunk));
  CK(c->cpb.ensure(sizeof(cpx<double>) * S * std::max(1, c->ngroup) * kProjChunk));
  CK(c->crb.ensure(sizeof(cpx<double>) * S * std::max(1, c->ngroup) * kProjChunk));
  CK(c->part.ensure(sizeof(double) * S * part_stride(c) * 4));
  CK(c->sysd.ensure(sizeof(double) * S * kSysD));
  CK(c->sysi.ensure(sizeof(int) * S * kSysI));
  CK(c->gpart.ensure(sizeof(double) * nb * gram_chunks(nd) * c->ns * c->ns));
  CK(c->cmat.ensure(cb * nb * c->ns * c->ns));
  CK(c->probe_d.ensure(sizeof(long long) * nb));
  CK(c->pomega_d.ensure(sizeof(double) * nb));
  CK(c->active_d.ensure(sizeof(int) * nb));
  CK(c->steps_d.ensure(sizeof(int) * nb));
  CK(c->alpha_d.ensure(sizeof(double) * nb * nl));
  CK(c->beta_d.ensure(sizeof(double) * nb * nl));
  CK(c->lstate_d.ensure(sizeof(double) * nb * 4));
  CK(c->coef_d.ensure(sizeof(double) * nb * (nl + 2)));
  CK(c->dots_d.ensure(sizeof(double) * nb * (nl + 2)));
  CK(c->dotpart_d.ensure(sizeof(double) * nb * 64 * (nl + 2)));
  CK(c->flags_d.ensure(sizeof(int) * 4));
  CK(c->dout_d.ensure(sizeof(double) * nb));
  CK(c->counts_d.ensure(sizeof(int) * kNumStatus * (1 + kChunkItersMax)));
  CK(c->list_d.ensure(sizeof(int) * S));
  c->ws_nb = nb;
  return RPA_OK;
}

// ---------------------------------------------------------------------------------------------
// statistics
// ---------------------------------------------------------------------------------------------
struct SolveStats {
  long long solves = 0, iters = 0, refine_rounds = 0;
  int max_iters = 0, nonconv = 0, breakdown = 0;
};

static rpa_status collect_stats(rpa_ctx* c, int S, SolveStats& ss) {
  std::vector<int> si((size_t)S * kSysI);
  CK(cudaMemcpyAsync(si.data(), c->sysi.p, sizeof(int) * S * kSysI, cudaMemcpyDeviceToHost,
                     c->stream));
  CK(cudaStreamSynchronize(c->stream));
  for (int s = 0; s < S; ++s) {
    const int st = si[(size_t)s * kSysI + kStatus];
    if (st == kIdle) continue;
    const int it = si[(size_t)s * kSysI + kIters];
    ss.solves += 1;
    ss.iters += it;
    ss.max_iters = std::max(ss.max_iters, it);
    ss.refine_rounds += si[(size_t)s * kSysI + kRestarts];
    if (st == kMaxit) ss.nonconv += 1;
    if (st == kBreakdown) ss.breakdown += 1;
  }
  return RPA_OK;
}

static rpa_status counts(rpa_ctx* c, int S, int* out, bool make_list = false) {
  CK(count_status(S, c->sysi.as<int>(), c->counts_d.as<int>(), c->stream,
                  make_list ? c->list_d.as<int>() : nullptr));
  CK(cudaMemcpyAsync(c->pinned, c->counts_d.p, sizeof(int) * kNumStatus, cudaMemcpyDeviceToHost,
                     c->stream));
  CK(cudaStreamSynchronize(c->stream));
  for (int i = 0; i < kNumStatus; ++i) out[i] = c->pinned[i];
  return RPA_OK;
}

// ---------------------------------------------------------------------------------------------
// Sternheimer solves for nb probe slots: dens_b = chi0(i w_b) u_b
// ---------------------------------------------------------------------------------------------
template <typename T>
static CocgView<T> make_view(rpa_ctx* c, int nb, const T* u, cpx<T>* x, cpx<T>* r, cpx<T>* p,
                             cpx<T>* w) {
  CocgView<T> cv;
  OpData<T>& o = opd<T>(c);
  cv.st = o.st;
  cv.vloc = o.vloc.template as<T>();
  cv.nl = nlview<T>(c);
  cv.nd = c->nd;
  cv.nsys = nb * c->ns;
  cv.ns = c->ns;
  cv.tiles = part_stride(c);
  cv.psi = o.psi.template as<T>();
  cv.eps = c->eps_d.as<double>();
  cv.omega = c->pomega_d.as<double>();
  cv.u = u;
  cv.x = x;
  cv.r = r;
  cv.p = p;
  cv.w = w;
  cv.cdot = c->cdot.as<cpx<T>>();
  cv.part = c->part.as<double>();
  cv.sysd = c->sysd.as<double>();
  cv.sysi = c->sysi.as<int>();
  cv.list = nullptr;
  return cv;
}

constexpr int kChunkIters = 4;
// smallest FP32 inner tolerance per refinement round at which the recurrence is continued
constexpr double kContinueMinInnerTol = 1e-3;
// Sternheimer tolerances at or above this use the double-float refinement residual
constexpr double kDfResidualTol = 1e-8;
static_assert(kChunkIters <= kChunkItersMax, "counts buffer holds one slot per iteration");
// with graphs and options.profile, one chunk in kProfEvery is launched directly with events
constexpr int kProfEvery = 4;
// with options.graphs = 2 and options.profile, one COCG loop in kProfLoopEvery is run
// host-checked (with its sample chunks) instead of as one graph
constexpr int kProfLoopEvery = 4;

template <typename T>
static FusedBufs<T> make_fused(rpa_ctx* c) {
  FusedBufs<T> fb;
  fb.p_in = c->p.as<cpx<T>>();
  fb.p_out = c->p2.as<cpx<T>>();
  fb.cp = c->cpb.as<cpx<T>>();
  fb.cr = c->crb.as<cpx<T>>();
  fb.tile_roff = c->tile_roff.as<int>();
  fb.tile_ranges = c->tile_ranges.as<int>();
  fb.ntiles_xy = fused_ntiles_xy(c);
  fb.nzchunk = fused_nzchunk(c);
  fb.zchunk = fused_zchunk(c);
  fb.tiles1d = (int)tiles_of(c->nd);
  fb.first = 1;
  fb.nact = 0;
  fb.row_ty = 0;
  fb.band_ty = 0;
  return fb;
}

// Tiling of a launch over `nact` systems: xy tiles of kind ty, and z split into chunks
// of at least R planes until the launch has about two waves of blocks on the GPU.
template <typename T>
static void set_tiling(const rpa_ctx* c, FusedBufs<T>& fb, int ty, int nact) {
  fb.row_ty = ty;
  fb.band_ty = is_band(ty) ? band_rows(ty) : 0;
  fb.ntiles_xy = is_band(ty) ? c->grid.n[1] / band_rows(ty)
                 : ty == kTileX2Packed ? x2p_tiles_xy(c->grid.n[0], c->grid.n[1])
                 : ty > 0    ? (c->grid.n[1] + ty - 1) / ty
                             : (is_x2(ty) ? x2_tiles_xy(c->grid.n[0], c->grid.n[1])
                                              : fused_ntiles_xy(c));
  const int nz = c->grid.n[2], R = c->grid.fd_radius;
  const int base = fused_zchunk(c);
  const long long want = 6LL * std::max(1, c->nsm);
  int zc = base;
  for (int f = 2; f <= kMaxZSplit; f *= 2) {
    const long long blocks = (long long)nact * fb.ntiles_xy * ((nz + zc - 1) / zc);
    const int next = (base + f - 1) / f;
    if (blocks >= want || next < R) break;
    zc = next;
  }
  fb.zchunk = zc;
  fb.nzchunk = (nz + zc - 1) / zc;
}

constexpr int kTailSystems = 32;  // launches over at most this many systems use the tail tiling

// Tiling of the H-apply kernel.  With options.tile = -1 every candidate (32 x 8 column
// tiles, 64 x 8 two-point tiles, each row-tile height row_candidates() lists) is timed on
// the systems of the first COCG loop of the precision — once over all of them (bulk) and
// once over the first few (tail) — and the fastest of each is kept for the context.  Timing
// runs the kernel in place: it reads r, p_{k-1} and the projector coefficients and writes
// p_k, w and its partial sums, all of which the first real iteration rewrites.
template <typename T>
static rpa_status choose_tiling(rpa_ctx* c, const CocgView<T>& cv, const FusedBufs<T>& fb,
                                int* ty_bulk, int* ty_tail) {
  const int k = sizeof(T) == 4 ? 0 : 1;
  if (c->opt.tile != -1) {
    *ty_bulk = *ty_tail = c->opt.tile;
    return RPA_OK;
  }
  if (c->tuned_ty[k][0] == -1) {
    int cand[32];
    int nc = 0;
    cand[nc++] = 0;
    if (sizeof(T) == 4 && x2_tile_fits(c->grid.n[0], c->grid.fd_radius)) {
      cand[nc++] = kTileX2;
      cand[nc++] = kTileX2Ring1;
      cand[nc++] = kTileX2Ring2;
    }
    if (sizeof(T) == 4) {
      int bty[8];
      const int nb = band_candidates(c->grid.n[0], c->grid.n[1], c->grid.fd_radius, c->ngroup,
                                     bty, 8);
      for (int i = 0; i < nb; ++i) cand[nc++] = band_code(bty[i]);
    }
    nc += row_candidates<T>(c->grid.n[0], c->grid.n[1], c->grid.fd_radius, c->ngroup, cand + nc,
                            std::min(16, 32 - nc));
    int best_ty[2] = {0, 0};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (nc > 1 && cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
      cudaError_t err = cudaSuccess;
      for (int regime = 0; regime < 2; ++regime) {
        FusedBufs<T> t = fb;
        t.first = 0;  // time the steady-state form (reads p_{k-1})
        t.nact = regime == 0 ? fb.nact : std::min(fb.nact, 8);
        float best = 1e30f;
        for (int i = 0; i < nc && err == cudaSuccess; ++i) {
          set_tiling(c, t, cand[i], t.nact);
          err = launch_dirmatvec_only<T>(cv, t, c->stream);  // warm-up
          if (err == cudaSuccess) err = cudaEventRecord(e0, c->stream);
          for (int rep = 0; rep < 3 && err == cudaSuccess; ++rep)
            err = launch_dirmatvec_only<T>(cv, t, c->stream);
          if (err == cudaSuccess) err = cudaEventRecord(e1, c->stream);
          if (err == cudaSuccess) err = cudaEventSynchronize(e1);
          float ms = 0.f;
          if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
          if (err == cudaSuccess && ms < best) {
            best = ms;
            best_ty[regime] = cand[i];
          }
        }
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      CK(err);
    } else if (e0) {
      cudaEventDestroy(e0);
    }
    c->tuned_ty[k][0] = best_ty[0];
    c->tuned_ty[k][1] = best_ty[1];
  }
  *ty_bulk = c->tuned_ty[k][0];
  *ty_tail = c->tuned_ty[k][1];
  return RPA_OK;
}

// One chunk of kChunkIters fused iterations as a CUDA graph.  Launch grids cover `bucket`
// systems (the next power of two above the active count, at most all systems); list entries
// past the active count are -1 and those blocks return at once, so one graph per bucket
// serves every chunk with that many or fewer active systems.  Graphs are cached on the
// context by the bytes of every launch parameter and replayed.  They hold no events: the
// profiling mode times directly launched sample chunks instead.
template <typename T>
static rpa_status run_chunk_graph(rpa_ctx* c, const CocgView<T>& cv, const FusedBufs<T>& fb,
                                  int maxit) {
  struct Key {
    int tsize, maxit;
    double tol;
    CocgView<T> cv;
    FusedBufs<T> fb;
  } k;
  std::memset(&k, 0, sizeof(k));  // padding bytes take part in the comparison
  k.tsize = (int)sizeof(T);
  k.maxit = maxit;
  k.tol = c->opt.stern_tol;
  k.cv = cv;
  k.fb = fb;
  const unsigned char* kb = reinterpret_cast<const unsigned char*>(&k);
  rpa_ctx::ChunkGraph* hit = nullptr;
  for (auto& g : c->graphs)
    if (g.key.size() == sizeof(k) && std::memcmp(g.key.data(), kb, sizeof(k)) == 0) {
      hit = &g;
      break;
    }
  if (!hit) {
    if (fb.row_ty > 0) CK(launch_dirmatvec_rows_prepare<T>());  // attributes before capture
    if (is_band(fb.row_ty)) CK(launch_dirmatvec_band_prepare());
    if (is_x2(fb.row_ty) && fb.row_ty != kTileX2) CK(launch_dirmatvec_x2_prepare());
    if (c->graphs.size() >= 64) {  // bounded cache: drop the oldest
      if (c->graphs.front().exec) cudaGraphExecDestroy(c->graphs.front().exec);
      c->graphs.erase(c->graphs.begin());
    }
    const long long l0 = rpa_kernel_launches(c);
    CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    FusedBufs<T> f = fb;
    cudaError_t err = cudaSuccess;
    for (int j = 0; j < kChunkIters && err == cudaSuccess; ++j) {
      err = fused_iteration<T>(cv, f, c->opt.stern_tol, maxit, c->stream, nullptr);
      std::swap(f.p_in, f.p_out);
      f.first = 0;
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t e_end = cudaStreamEndCapture(c->stream, &graph);
    const int nl = (int)(rpa_kernel_launches(c) - l0);
    note_launch(-nl);  // captured, not launched
    if (err == cudaSuccess) err = e_end;
    cudaGraphExec_t exec = nullptr;
    if (err == cudaSuccess) err = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    CK(err);
    c->graphs.emplace_back();
    c->graphs.back().key.assign(kb, kb + sizeof(k));
    c->graphs.back().exec = exec;
    c->graphs.back().launches = nl;
    hit = &c->graphs.back();
  }
  CK(cudaGraphLaunch(hit->exec, c->stream));
  note_launch(hit->launches);
  return RPA_OK;
}

// The whole COCG loop as one CUDA graph, with no host check between chunks (options.graphs
// = 2).  Launch widths are the power-of-two buckets of the host-checked loop: a prologue
// chunk (the first iteration starts the recurrence) over W_0 systems, then one level per
// width W_0 > W_1 > ... > 1, each a while node that repeats its chunk over W_i systems as
// long as more than W_{i+1} are active.  After every chunk the active list and counts are
// rebuilt on the device and a one-thread kernel sets the level's condition.  An iteration
// counter bounds every level (the per-system cap marks every system by maxit + 2 chunks),
// so each loop ends even if no status changes.  Graphs are cached like the chunk graphs.
template <typename T>
static rpa_status run_loop_graph(rpa_ctx* c, const CocgView<T>& cv, const FusedBufs<T>& fb,
                                 int maxit, int ty_bulk, int ty_tail) {
  const int nsys = cv.nsys;
  int w0 = 1;
  while (w0 < fb.nact) w0 <<= 1;
  w0 = std::min(w0, nsys);
  std::vector<int> widths{w0};
  {
    int w = 1;
    while (w < w0) w <<= 1;
    for (w >>= 1; w >= 1; w >>= 1) widths.push_back(w);
  }
  struct Key {
    int kind, tsize, maxit, w0, ty_bulk, ty_tail;
    double tol;
    CocgView<T> cv;
    FusedBufs<T> fb;
  } k;
  std::memset(&k, 0, sizeof(k));  // padding bytes take part in the comparison
  k.kind = 2;
  k.tsize = (int)sizeof(T);
  k.maxit = maxit;
  k.w0 = w0;
  k.ty_bulk = ty_bulk;
  k.ty_tail = ty_tail;
  k.tol = c->opt.stern_tol;
  k.cv = cv;
  k.fb = fb;
  k.fb.nact = 0;
  const unsigned char* kb = reinterpret_cast<const unsigned char*>(&k);
  rpa_ctx::ChunkGraph* hit = nullptr;
  for (auto& g : c->graphs)
    if (g.key.size() == sizeof(k) && std::memcmp(g.key.data(), kb, sizeof(k)) == 0) {
      hit = &g;
      break;
    }
  CK(c->loopctl_d.ensure(2 * sizeof(unsigned long long)));
  unsigned long long* ctl = c->loopctl_d.as<unsigned long long>();
  int* cnts = c->counts_d.as<int>();
  if (!hit) {
    for (int ty : {ty_bulk, ty_tail}) {  // kernel attributes before capture
      if (ty > 0) CK(launch_dirmatvec_rows_prepare<T>());
      if (is_band(ty)) CK(launch_dirmatvec_band_prepare());
      if (is_x2(ty) && ty != kTileX2) CK(launch_dirmatvec_x2_prepare());
    }
    if (c->graphs.size() >= 64) {  // bounded cache: drop the oldest
      if (c->graphs.front().exec) cudaGraphExecDestroy(c->graphs.front().exec);
      c->graphs.erase(c->graphs.begin());
    }
    const long long l0 = rpa_kernel_launches(c);
    const int limit = maxit + 2 * kChunkIters;
    const cudaStreamCaptureMode mode = cudaStreamCaptureModeThreadLocal;
    // chunk of kChunkIters iterations over `width` systems (an even count: p_in / p_out end
    // as they started), then the active list and counts
    auto chunk = [&](cudaStream_t s, int width, int first) -> cudaError_t {
      FusedBufs<T> g = fb;
      g.nact = width;
      set_tiling(c, g, width <= kTailSystems ? ty_tail : ty_bulk, width);
      g.first = first;
      for (int j = 0; j < kChunkIters; ++j) {
        const cudaError_t e = fused_iteration<T>(cv, g, c->opt.stern_tol, maxit, s, nullptr);
        if (e != cudaSuccess) return e;
        std::swap(g.p_in, g.p_out);
        g.first = 0;
      }
      return count_status(nsys, cv.sysi, cnts, s, c->list_d.as<int>());
    };
    // capture fn's launches into graph g after node dep (none if null); *last = its last node
    auto segment = [&](cudaGraph_t g, cudaGraphNode_t dep, auto&& fn,
                       cudaGraphNode_t* last) -> cudaError_t {
      cudaError_t e = cudaStreamBeginCaptureToGraph(c->stream, g, dep ? &dep : nullptr, nullptr,
                                                    dep ? 1 : 0, mode);
      if (e != cudaSuccess) return e;
      const cudaError_t ef = fn(c->stream);
      cudaStreamCaptureStatus cs;
      const cudaGraphNode_t* deps = nullptr;
      size_t nd = 0;
      const cudaError_t ei =
          cudaStreamGetCaptureInfo(c->stream, &cs, nullptr, nullptr, &deps, nullptr, &nd);
      if (last) *last = (ei == cudaSuccess && nd == 1) ? deps[0] : nullptr;
      cudaGraph_t out = g;
      const cudaError_t ee = cudaStreamEndCapture(c->stream, &out);
      if (ef != cudaSuccess) return ef;
      if (ei != cudaSuccess) return ei;
      if (ee != cudaSuccess) return ee;
      return (last && nd != 1) ? cudaErrorStreamCaptureUnjoined : cudaSuccess;
    };
    cudaGraph_t parent = nullptr;
    cudaError_t err = cudaGraphCreate(&parent, 0);
    cudaGraphNode_t tail = nullptr;
    int parent_launches = 0;
    if (err == cudaSuccess)
      err = segment(parent, nullptr, [&](cudaStream_t s) -> cudaError_t {
        cudaError_t e = cudaMemsetAsync(ctl, 0, 2 * sizeof(unsigned long long), s);
        if (e == cudaSuccess) e = chunk(s, w0, fb.first);
        return e;
      }, &tail);
    parent_launches = (int)(rpa_kernel_launches(c) - l0);
    for (size_t i = 0; i < widths.size() && err == cudaSuccess; ++i) {
      const int wnext = i + 1 < widths.size() ? widths[i + 1] : 0;
      // the prologue's iterations are counted by the first level's check
      const int add = i == 0 ? kChunkIters : 0;
      cudaGraphConditionalHandle h;
      // default 0 at every launch: a level whose check did not run is skipped, never spun
      err = cudaGraphConditionalHandleCreate(&h, parent, 0, cudaGraphCondAssignDefault);
      if (err != cudaSuccess) break;
      const long long lp = rpa_kernel_launches(c);
      err = segment(parent, tail, [&](cudaStream_t s) {
        return loop_cond(cnts, ctl, h, wnext, limit, add, 0, s);
      }, &tail);
      parent_launches += (int)(rpa_kernel_launches(c) - lp);
      if (err != cudaSuccess) break;
      cudaGraphNodeParams np = {};
      np.type = cudaGraphNodeTypeConditional;
      np.conditional.handle = h;
      np.conditional.type = cudaGraphCondTypeWhile;
      np.conditional.size = 1;
      cudaGraphNode_t wn = nullptr;
      err = cudaGraphAddNode(&wn, parent, &tail, nullptr, 1, &np);
      if (err != cudaSuccess) break;
      cudaGraph_t body = np.conditional.phGraph_out[0];
      const int width = widths[i];
      err = segment(body, nullptr, [&](cudaStream_t s) -> cudaError_t {
        const long long lb = rpa_kernel_launches(c);
        cudaError_t e = chunk(s, width, 0);
        if (e != cudaSuccess) return e;
        const int nb = (int)(rpa_kernel_launches(c) - lb) + 1;  // and the check itself
        return loop_cond(cnts, ctl, h, wnext, limit, kChunkIters, nb, s);
      }, nullptr);
      tail = wn;
    }
    note_launch(-(int)(rpa_kernel_launches(c) - l0));  // captured, not launched
    cudaGraphExec_t exec = nullptr;
    if (err == cudaSuccess) err = cudaGraphInstantiate(&exec, parent, 0);
    if (parent) cudaGraphDestroy(parent);
    CK(err);
    c->graphs.emplace_back();
    c->graphs.back().key.assign(kb, kb + sizeof(k));
    c->graphs.back().exec = exec;
    c->graphs.back().launches = parent_launches;
    hit = &c->graphs.back();
  }
  CK(cudaGraphLaunch(hit->exec, c->stream));
  unsigned long long hctl[2] = {0, 0};
  CK(cudaMemcpyAsync(hctl, ctl, sizeof(hctl), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  note_launch(hit->launches + (int)hctl[1]);
  return RPA_OK;
}

// COCG iterations until no system is active.  Expects r (and x) set for the active systems;
// forms the projector coefficients of r, then iterates the fused kernels.  With cont, the
// recurrence continues from the direction kept in p (and its projector coefficients in cp)
// with the beta each system holds, instead of starting from p = r.
template <typename T>
static rpa_status cocg_loop(rpa_ctx* c, const CocgView<T>& cv_all, int maxit, bool cont = false) {
  int cnt[kNumStatus];
  int done_iters = 0;
  const bool prof = c->opt.profile && c->have_pev && c->prof_stats;
  FusedBufs<T> fb = make_fused<T>(c);
  CK(proj_dots<T>(cv_all.nl, cv_all.nd, cv_all.nsys, cv_all.r, cv_all.sysi, 1 << kActive, fb.cr,
                  c->stream));
  CK(fused_prepare<T>(cv_all, fb, c->stream, cont ? 0 : 1));
  if (cont) fb.first = 0;
  // launches cover only the active systems, listed at every chunk boundary
  CocgView<T> cv = cv_all;
  cv.list = c->list_d.as<int>();
  CKS(counts(c, cv_all.nsys, cnt, true));
  fb.nact = cnt[kActive];
  int ty_bulk = 0, ty_tail = 0;
  if (fb.nact > 0) CKS(choose_tiling<T>(c, cv, fb, &ty_bulk, &ty_tail));
  if (c->prof_stats) {
    c->prof_stats->tile_rows = ty_bulk;
    c->prof_stats->tile_rows_tail = ty_tail;
  }
  const bool graphs = c->opt.graphs != 0;
  // graphs = 2: the whole loop on the device; with profiling, every kProfLoopEvery-th loop
  // runs host-checked instead, its sample chunks timed with events
  if (c->opt.graphs == 2 && fb.nact > 0 && !(prof && c->loop_no++ % kProfLoopEvery == 0))
    return run_loop_graph<T>(c, cv, fb, maxit, ty_bulk, ty_tail);
  const size_t cpxb = sizeof(cpx<T>);
  int chunk_no = 0;
  while (fb.nact > 0) {
    // profiled chunk: kernels launched one by one between events, with the active count
    // recorded before each iteration for the algorithmic bytes of exactly these launches
    const bool sample = prof && (!graphs || chunk_no % kProfEvery == 0);
    int width = fb.nact;  // systems a launch covers
    if (graphs && !sample) {
      int bucket = 1;
      while (bucket < fb.nact) bucket <<= 1;
      width = std::min(bucket, cv_all.nsys);
    }
    FusedBufs<T> g = fb;
    g.nact = width;
    set_tiling(c, g, width <= kTailSystems ? ty_tail : ty_bulk, width);
    if (graphs && !sample) {
      CKS(run_chunk_graph<T>(c, cv, g, maxit));
    } else {
      for (int j = 0; j < kChunkIters; ++j) {
        if (sample)
          CK(count_status(cv_all.nsys, cv_all.sysi, c->counts_d.as<int>() + kNumStatus * (1 + j),
                          c->stream, nullptr));
        CK(fused_iteration<T>(cv, g, c->opt.stern_tol, maxit, c->stream,
                              sample ? c->pev + 7 * j : nullptr));
        std::swap(g.p_in, g.p_out);
        g.first = 0;
      }
    }
    fb.first = 0;  // an even number of iterations leaves p_in / p_out as they were
    ++chunk_no;
    done_iters += kChunkIters;
    if (sample)  // the per-iteration counts, read with the chunk-end counts below
      CK(cudaMemcpyAsync(c->pinned + kNumStatus, c->counts_d.as<int>() + kNumStatus,
                         sizeof(int) * kNumStatus * kChunkIters, cudaMemcpyDeviceToHost,
                         c->stream));
    CKS(counts(c, cv_all.nsys, cnt, true));  // synchronises: the events are complete
    if (sample) {
      rpa_stats* st = c->prof_stats;
      const int part = width <= kTailSystems ? 5 : 6;  // tail / bulk chunk
      for (int j = 0; j < kChunkIters; ++j) {
        // interval (i, i+1) of iteration j -> kernel class
        static const int cls[6] = {0, 1, 2, 3, 2, 4};
        for (int i = 0; i < 6; ++i) {
          float ms = 0.f;
          CK(cudaEventElapsedTime(&ms, c->pev[7 * j + i], c->pev[7 * j + i + 1]));
          st->kernel_seconds[cls[i]] += 1e-3 * ms;
          st->kernel_seconds[part] += 1e-3 * ms;
          st->kernel_launches[cls[i]] += (i == 1 || i == 3) ? 1 : 0;
        }
        st->kernel_launches[part] += 1;
        const double pts = (double)c->pinned[kNumStatus * (1 + j) + kActive] * (double)c->nd;
        st->kernel_bytes[1] += pts * 4.0 * cpxb;  // direction + H apply: read r, p; write p, w
        st->kernel_bytes[3] += pts * 6.0 * cpxb;  // update: read x, p, r, w; write x, r
      }
      st->precision_bytes = (int)(cpxb / 2);
    }
    fb.nact = cnt[kActive];
    if (done_iters > maxit + 2 * kChunkIters) break;  // every system is marked by then
  }
  return RPA_OK;
}

// FP64 form: Galerkin guess, COCG, true-residual recheck at exit with a restart while it is
// above the tolerance.
static rpa_status solve_fp64(rpa_ctx* c, int nb, const double* u, const int* active,
                             SolveStats& ss) {
  const int S = nb * c->ns;
  const int maxit = c->opt.stern_maxit;
  cpx<double>*x = c->x.as<cpx<double>>(), *r = c->r.as<cpx<double>>(),
             *p = c->p.as<cpx<double>>(), *w = c->w.as<cpx<double>>();
  CocgView<double> cv = make_view<double>(c, nb, u, x, r, p, w);
  CK(galerkin_guess<double>(c->nd, c->ns, nb, c->d64.psi.as<double>(), c->eps_d.as<double>(),
                            c->pomega_d.as<double>(), u, active, c->dV, c->gpart.as<double>(),
                            gram_chunks(c->nd), c->cmat.as<cpx<double>>(), x, c->stream));
  CK(set_status(S, c->ns, active, kActive, c->sysi.as<int>(), c->stream));
  CK(proj_dots<double>(cv.nl, c->nd, S, x, cv.sysi, 1 << kActive, cv.cdot, c->stream));
  CK((cocg_resid<double, double>(cv, x, r, p, 1 << kActive, nullptr, nullptr, nullptr,
                                 c->stream)));
  CK(cocg_scalars(S, cv.tiles, cv.part, cv.sysd, cv.sysi, 0, 1 << kActive, c->opt.stern_tol, 0.0,
                  maxit, 0, c->stream));
  for (int round = 0; round < 60; ++round) {
    CKS(cocg_loop<double>(c, cv, maxit));
    int cnt[kNumStatus];
    CKS(counts(c, S, cnt));
    if (cnt[kConverged] == 0) break;
    // true residual of recursively converged systems; restart those above tolerance
    CK(proj_dots<double>(cv.nl, c->nd, S, x, cv.sysi, 1 << kConverged, cv.cdot, c->stream));
    CK((cocg_resid<double, double>(cv, x, r, p, 1 << kConverged, nullptr, nullptr, nullptr,
                                   c->stream)));
    CK(cocg_scalars(S, cv.tiles, cv.part, cv.sysd, cv.sysi, 3, 1 << kConverged,
                    c->opt.stern_tol, 0.0, maxit, 50, c->stream));
    CKS(counts(c, S, cnt));
    if (cnt[kActive] == 0) break;
  }
  CKS(collect_stats(c, S, ss));
  CK((density<double, double>(c->nd, c->ns, nb, c->d64.psi.as<double>(), x, active,
                              c->dens64.as<double>(), c->stream)));
  return RPA_OK;
}

// Mixed form: FP32 Galerkin guess and COCG; FP64 residual refinement rounds solve for FP32
// corrections that are accumulated in FP64.
static rpa_status solve_mixed(rpa_ctx* c, int nb, const float* u32, const int* active,
                              SolveStats& ss) {
  const int S = nb * c->ns;
  const int maxit = c->opt.stern_maxit;
  const double tol = c->opt.stern_tol;
  // FP32 rounds aim at sqrt(tol) (>= 1e-5): short rounds keep the FP32 recurrence in its
  // accurate regime; FP64 residuals restart them until tol is met.
  const double itol = c->opt.inner_tol > 0.0
                          ? c->opt.inner_tol
                          : (c->opt.refine > 0 ? std::max(std::sqrt(tol), 1e-5) : tol);
  cpx<float>*x = c->x.as<cpx<float>>(), *r = c->r.as<cpx<float>>(), *p = c->p.as<cpx<float>>(),
            *w = c->w.as<cpx<float>>();
  CocgView<float> cv = make_view<float>(c, nb, u32, x, r, p, w);
  CK(galerkin_guess_tc(c->nd, c->ns, nb, c->d32.psi.as<float>(), c->eps_d.as<double>(),
                       c->pomega_d.as<double>(), u32, active, c->dV, c->gpart.as<double>(),
                       gram_chunks(c->nd), c->cmat.as<cpx<float>>(), x, c->flags_d.as<int>() + 2,
                       c->stream, c->opt.precision == RPA_MIXED_BF16,
                       c->opt.debug_expire_waits));
  CK(set_status(S, c->ns, active, kActive, c->sysi.as<int>(), c->stream));
  CK(proj_dots<float>(cv.nl, c->nd, S, x, cv.sysi, 1 << kActive, cv.cdot, c->stream));
  CK((cocg_resid<float, float>(cv, x, r, p, 1 << kActive, nullptr, nullptr, nullptr, c->stream)));
  CK(cocg_scalars(S, cv.tiles, cv.part, cv.sysd, cv.sysi, 5, 1 << kActive, tol, itol, maxit, 0,
                  c->stream));
  CKS(cocg_loop<float>(c, cv, maxit));
  if (c->opt.refine <= 0) {
    CKS(collect_stats(c, S, ss));
    CK((density<float, float>(c->nd, c->ns, nb, c->d32.psi.as<float>(), x, active,
                              c->dens64.as<double>(), c->stream)));
    return RPA_OK;
  }
  // FP64 refinement.  The accumulated solution is kept as double-float pairs (hi, lo) of
  // each component; the residual runs in double-float arithmetic on the FP32 units while
  // the tolerance leaves room for its ~2^-48 rounding, else in FP64.
  float4* x64 = c->x64.as<float4>();
  cpx<double>* x64v = c->x64.as<cpx<double>>();  // the same storage, as the FP64 view's x
  const int all_but_idle = ((1 << kNumStatus) - 1) & ~(1 << kIdle);
  CK(accumulate_df(c->nd, S, c->sysi.as<int>(), all_but_idle, -1, x, x64, 1, c->stream));
  CK(convert_f2d(u32, c->u64.as<double>(), (long long)nb * c->nd, c->stream));
  CK(convert_d2df(c->u64.as<double>(), c->u2.as<float2>(), (long long)nb * c->nd, c->stream));
  CocgView<double> cv64 = make_view<double>(c, nb, c->u64.as<double>(), x64v, nullptr, nullptr,
                                            nullptr);
  DfAux aux;
  aux.nl = nlview<float>(c);
  aux.g_chi_lo = c->g_chi_lo.as<float>();
  aux.p_chi_lo = c->p_chi_lo.as<float>();
  aux.coef_lo = c->coef_lo.as<float>();
  aux.vloc = c->vloc2.as<float2>();
  aux.psi = c->psi2.as<float2>();
  aux.u = c->u2.as<float2>();
  const bool use_df = tol >= kDfResidualTol;
  // Each round replaces the FP32 recursive residual by the FP64 true residual.  By default
  // the FP32 recurrence then continues from its last direction (a reliable update: the
  // Krylov space built so far is kept) as long as a round reduces the residual by at most
  // kContinueMinInnerTol: deeper FP32 rounds leave rounding in the kept direction that is
  // large next to the new residual, and the continued recurrence stalls (measured at an
  // inner tolerance of 1e-5).  Otherwise, or with refine_restart = 1, each round restarts
  // from p = r.
  const bool cont = c->opt.refine_restart == 0 && itol >= kContinueMinInnerTol;
  bool rounds_left = false;  // the last round ran: its corrections are not checked yet
  for (int round = 1; round <= c->opt.refine; ++round) {
    rounds_left = false;
    CK(proj_dots_df(aux, c->nd, S, x64, cv64.sysi, 1 << kConverged, cv64.cdot, c->stream));
    CK((cocg_resid<double, float>(cv64, x64v, nullptr, nullptr, 1 << kConverged, r, p, x,
                                  c->stream, use_df, cont ? c->p2.as<cpx<float>>() : nullptr,
                                  &aux)));
    CK(cocg_scalars(S, cv64.tiles, cv64.part, cv64.sysd, cv64.sysi, cont ? 6 : 4,
                    1 << kConverged, tol, itol, maxit, 0, c->stream));
    int cnt[kNumStatus];
    CKS(counts(c, S, cnt));
    if (cnt[kActive] == 0) break;
    CKS(cocg_loop<float>(c, cv, maxit, cont));
    const int corrected = (1 << kConverged) | (1 << kMaxit) | (1 << kBreakdown);
    CK(accumulate_df(c->nd, S, c->sysi.as<int>(), corrected, round, x, x64, 0, c->stream));
    // systems that were final before this round keep status kFinal and are skipped above;
    // systems corrected this round are kConverged again and are re-checked next round.
    rounds_left = true;
  }
  if (rounds_left) {
    // the rounds are used up: check the last corrections in FP64, so that a system still
    // above the tolerance is reported (not converged) instead of passing silently
    int cnt[kNumStatus];
    CKS(counts(c, S, cnt));
    if (cnt[kConverged] > 0) {
      CK(proj_dots_df(aux, c->nd, S, x64, cv64.sysi, 1 << kConverged, cv64.cdot, c->stream));
      CK((cocg_resid<double, float>(cv64, x64v, nullptr, nullptr, 1 << kConverged, nullptr,
                                    nullptr, nullptr, c->stream, use_df, nullptr, &aux)));
      CK(cocg_scalars(S, cv64.tiles, cv64.part, cv64.sysd, cv64.sysi, 7, 1 << kConverged, tol,
                      itol, maxit, 0, c->stream));
    }
  }
  CKS(collect_stats(c, S, ss));
  CK((density_df(c->nd, c->ns, nb, c->d64.psi.as<double>(), x64, active,
                              c->dens64.as<double>(), c->stream)));
  return RPA_OK;
}

// ---------------------------------------------------------------------------------------------
// one wave of nb probe-points: Lanczos quadrature (Algorithm 1, inner part)
// ---------------------------------------------------------------------------------------------
struct WaveOut {
  double* d;      // host, nb
  double* alpha;  // host, nb x nl (may be null)
  double* beta;
  int* steps;
};

static rpa_status timing_mark(rpa_ctx* c, int i) {
  if (c->have_events) CK(cudaEventRecord(c->ev[i], c->stream));
  return RPA_OK;
}

static rpa_status timing_add(rpa_ctx* c, rpa_stats* st, int from, int to, int phase) {
  if (!c->have_events || !st) return RPA_OK;
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, c->ev[from], c->ev[to]));
  st->seconds_phase[phase] += 1e-3 * ms;
  return RPA_OK;
}

// Block layout of a wave for block Lanczos: slot s belongs to the block of consecutive slots
// starting at first[s] with size[s] members (all one frequency, distinct points).
struct BlockLayout {
  std::vector<int> first, size;  // per slot
  std::vector<int> start, sz;    // per block
};

static rpa_status run_wave(rpa_ctx* c, int nb, const long long* probe_h, const double* omega_h,
                           WaveOut out, rpa_stats* st, const BlockLayout* blk = nullptr) {
  const long long nd = c->nd;
  const int nl = c->opt.lanczos_max;
  const long long ldq = (long long)(nl + 1) * nd;
  const bool mixed = c->opt.precision != RPA_FP64;
  double* Q = c->Q.as<double>();
  int* active = c->active_d.as<int>();
  CK(cudaMemcpyAsync(c->probe_d.p, probe_h, sizeof(long long) * nb, cudaMemcpyHostToDevice,
                     c->stream));
  CK(cudaMemcpyAsync(c->pomega_d.p, omega_h, sizeof(double) * nb, cudaMemcpyHostToDevice,
                     c->stream));
  {
    std::vector<int> ones(nb, 1);
    CK(cudaMemcpyAsync(active, ones.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  CK(cudaMemsetAsync(c->alpha_d.p, 0, sizeof(double) * nb * nl, c->stream));
  CK(cudaMemsetAsync(c->beta_d.p, 0, sizeof(double) * nb * nl, c->stream));
  CK(cudaMemsetAsync(c->steps_d.p, 0, sizeof(int) * nb, c->stream));
  CK(cudaMemsetAsync(c->lstate_d.p, 0, sizeof(double) * nb * 4, c->stream));
  CK(cudaMemsetAsync(c->flags_d.p, 0, sizeof(int) * 4, c->stream));
  CK(lanczos_start(nd, nb, c->probe_d.as<long long>(), Q, ldq, c->stream));
  const int nchunk = (int)std::max<long long>(1, std::min<long long>(64, (nd + 8191) / 8192));
  double* dots = c->dots_d.as<double>();
  double* dpart = c->dotpart_d.as<double>();
  double* coef = c->coef_d.as<double>();
  double* v = c->v64.as<double>();
  const int bmax = c->opt.lanczos_block;
  const int nblk = blk ? (int)blk->start.size() : 0;
  int *bfirst = nullptr, *bsize = nullptr, *bstart = nullptr, *bsz = nullptr, *bsteps = nullptr;
  const long long ldT = (long long)nl * bmax * nl * bmax, ldl = (long long)nl * bmax;
  if (blk) {
    const size_t ntj = (size_t)bmax * (nl + 1);
    CK(c->bD.ensure(sizeof(double) * nb * ntj));
    CK(c->bpart.ensure(sizeof(double) * nb * ntj * nchunk));
    CK(c->bA.ensure(sizeof(double) * nblk * nl * 64));
    CK(c->bB.ensure(sizeof(double) * nblk * nl * 64));
    CK(c->bR.ensure(sizeof(double) * nblk * 64));
    CK(c->bRinv.ensure(sizeof(double) * nblk * 64));
    CK(c->bT.ensure(sizeof(double) * nblk * ldT));
    CK(c->bW.ensure(sizeof(double) * nblk * ldT));
    CK(c->blam.ensure(sizeof(double) * nblk * ldl));
    CK(c->bsteps.ensure(sizeof(int) * nblk));
    CK(c->bm.ensure(sizeof(int) * nblk));
    CK(c->bfirst.ensure(sizeof(int) * nb));
    CK(c->bsize.ensure(sizeof(int) * nb));
    CK(c->bstart.ensure(sizeof(int) * nblk));
    CK(c->bsz.ensure(sizeof(int) * nblk));
    bfirst = c->bfirst.as<int>();
    bsize = c->bsize.as<int>();
    bstart = c->bstart.as<int>();
    bsz = c->bsz.as<int>();
    bsteps = c->bsteps.as<int>();
    CK(cudaMemcpyAsync(bfirst, blk->first.data(), sizeof(int) * nb, cudaMemcpyHostToDevice,
                       c->stream));
    CK(cudaMemcpyAsync(bsize, blk->size.data(), sizeof(int) * nb, cudaMemcpyHostToDevice,
                       c->stream));
    CK(cudaMemcpyAsync(bstart, blk->start.data(), sizeof(int) * nblk, cudaMemcpyHostToDevice,
                       c->stream));
    CK(cudaMemcpyAsync(bsz, blk->sz.data(), sizeof(int) * nblk, cudaMemcpyHostToDevice,
                       c->stream));
    CK(cudaMemsetAsync(bsteps, 0, sizeof(int) * nblk, c->stream));
    CK(cudaStreamSynchronize(c->stream));  // the host vectors may go away
  }
  int steps_done = 0;
  for (int k = 0; k < nl; ++k) {
    SolveStats ss;
    CKS(timing_mark(c, 0));
    // u = nu^{1/2} q_k
    if (mixed) {
      CKS((nu_half<float, double, float>(c, Q + (long long)k * nd, ldq, c->u32.as<float>(), nb,
                                         c->t32a.as<float>(), c->t32b.as<float>())));
    } else {
      CKS((nu_half<double, double, double>(c, Q + (long long)k * nd, ldq, c->u64.as<double>(), nb,
                                           c->t64a.as<double>(), c->t64b.as<double>())));
    }
    CKS(timing_mark(c, 1));
    // Sternheimer solves and density (Galerkin guess + COCG)
    if (mixed)
      CKS(solve_mixed(c, nb, c->u32.as<float>(), active, ss));
    else
      CKS(solve_fp64(c, nb, c->u64.as<double>(), active, ss));
    CKS(timing_mark(c, 2));
    // v = nu^{1/2} r
    if (mixed) {
      CKS((nu_half<float, double, double>(c, c->dens64.as<double>(), nd, v, nb,
                                          c->t32a.as<float>(), c->t32b.as<float>())));
    } else {
      CKS((nu_half<double, double, double>(c, c->dens64.as<double>(), nd, v, nb,
                                           c->t64a.as<double>(), c->t64b.as<double>())));
    }
    CKS(timing_mark(c, 3));
    if (blk) {
      // block step: projections on every previous block (two classical Gram-Schmidt passes,
      // the first also giving the diagonal block A_k), then Cholesky QR twice -> Q_{k+1}, B_k
      const int nj = k + 1, ldD = bmax * nj;
      double* D = c->bD.as<double>();
      for (int pass = 0; pass < 2; ++pass) {
        CK(block_dot(nd, nb, bmax, bfirst, bsize, Q, ldq, nd, 0, nj, v, active,
                     c->bpart.as<double>(), nchunk, D, c->stream));
        if (pass == 0)
          CK(block_store_a(nblk, bstart, bsz, D, ldD, nj, k, nl, c->bA.as<double>(), active,
                           c->stream));
        CK(block_axpy(nd, nb, bfirst, bsize, Q, ldq, nj, D, ldD, v, active, c->stream));
      }
      if (k + 1 < nl) {
        for (int pass = 0; pass < 2; ++pass) {
          CK(block_dot(nd, nb, bmax, bfirst, bsize, v, nd, nd, 0, 1, v, active,
                       c->bpart.as<double>(), nchunk, D, c->stream));
          CK(block_chol(nblk, bstart, bsz, D, bmax, pass, k, nl, c->bA.as<double>(),
                        c->bR.as<double>(), c->bRinv.as<double>(), c->bB.as<double>(), active,
                        bsteps, c->stream));
          CK(block_scale(nd, nblk, bstart, bsz, c->bRinv.as<double>(), v,
                         pass == 0 ? v : Q + (long long)(k + 1) * nd, pass == 0 ? nd : ldq,
                         active, c->stream));
        }
      }
      steps_done = k + 1;
    } else {
      // alpha_k = q_k^T v ; v -= alpha_k q_k + beta_{k-1} q_{k-1}
      CK(multi_dot(nd, nb, Q, ldq, k, k + 1, v, active, dpart, nchunk, dots, c->stream));
      CK(lanczos_alpha(nb, k, nl, dots, active, c->alpha_d.as<double>(), c->beta_d.as<double>(),
                       coef, c->stream));
      CK(multi_axpy(nd, nb, Q, ldq, std::max(0, k - 1), k + 1, k > 0 ? coef : coef + 1, 2, v,
                    active, c->stream));
      if (c->opt.reorth) {
        for (int pass = 0; pass < 2; ++pass) {
          CK(multi_dot(nd, nb, Q, ldq, 0, k + 1, v, active, dpart, nchunk, dots, c->stream));
          CK(multi_axpy(nd, nb, Q, ldq, 0, k + 1, dots, k + 1, v, active, c->stream));
        }
      }
      // beta_k = ||v||, q_{k+1} = v / beta_k (with breakdown / early-exit tests)
      CK(multi_dot(nd, nb, v, nd, 0, 1, v, active, dpart, nchunk, dots, c->stream));
      CK(lanczos_beta(nb, k, nl, dots, active, c->alpha_d.as<double>(), c->beta_d.as<double>(),
                      c->steps_d.as<int>(), c->lstate_d.as<double>(), c->opt.lanczos_rtol,
                      c->opt.fkind, c->flags_d.as<int>(), c->stream));
      CK(lanczos_next(nd, nb, k, nl, active, c->lstate_d.as<double>(), c->beta_d.as<double>(), v, Q,
                      ldq, c->stream));
    }
    CKS(timing_mark(c, 4));
    // stats and the number of probes still running
    std::vector<int> act(nb);
    CK(cudaMemcpyAsync(act.data(), active, sizeof(int) * nb, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (st) {
      st->solves += ss.solves;
      st->nonconv_solves += ss.nonconv;
      st->breakdown_solves += ss.breakdown;
      st->cocg_iters += ss.iters;
      st->refine_rounds += ss.refine_rounds;
      st->max_cocg_iters = std::max(st->max_cocg_iters, ss.max_iters);
      CKS(timing_add(c, st, 0, 1, 0));
      CKS(timing_add(c, st, 1, 2, 2));
      CKS(timing_add(c, st, 2, 3, 0));
      CKS(timing_add(c, st, 3, 4, 4));
    }
    if (ss.nonconv) note_soft(c, RPA_ENOCONV, "a Sternheimer solve reached stern_maxit");
    if (ss.breakdown)
      note_soft(c, RPA_EBREAKDOWN,
                "a COCG solve broke down (p^T A p = 0 or a non-finite residual)");
    int any = 0;
    for (int b = 0; b < nb; ++b) any += act[b];
    // one matrix-vector product per probe-point that ran this step
    if (st) st->matvecs += (long long)(ss.solves / std::max(1, c->ns));
    // a non-converged or broken-down solve is recorded in c->err; the step's results stand
    if (any == 0) break;
  }
  CKS(timing_mark(c, 5));
  if (blk) {
    CK(block_quadrature(nblk, bstart, bsz, bsteps, steps_done, nl, c->bA.as<double>(),
                        c->bB.as<double>(), c->bT.as<double>(), c->bW.as<double>(),
                        c->blam.as<double>(), ldT, ldl, c->bm.as<int>(), c->opt.fkind,
                        c->dout_d.as<double>(), c->stream));
    // per-slot step counts from the blocks
    std::vector<int> bs(nblk), per(nb);
    CK(cudaMemcpyAsync(bs.data(), bsteps, sizeof(int) * nblk, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int B = 0; B < nblk; ++B)
      for (int l = 0; l < blk->sz[B]; ++l)
        per[blk->start[B] + l] = bs[B] > 0 ? bs[B] : steps_done;
    CK(cudaMemcpyAsync(c->steps_d.p, per.data(), sizeof(int) * nb, cudaMemcpyHostToDevice,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
  } else {
    CK(tridiag_f11(nb, nl, c->alpha_d.as<double>(), nl, c->beta_d.as<double>(), nl,
                   c->steps_d.as<int>(), c->opt.fkind, c->dout_d.as<double>(), c->stream));
  }
  CKS(timing_mark(c, 6));
  CK(cudaMemcpyAsync(out.d, c->dout_d.p, sizeof(double) * nb, cudaMemcpyDeviceToHost, c->stream));
  if (out.alpha)
    CK(cudaMemcpyAsync(out.alpha, c->alpha_d.p, sizeof(double) * nb * nl, cudaMemcpyDeviceToHost,
                       c->stream));
  if (out.beta)
    CK(cudaMemcpyAsync(out.beta, c->beta_d.p, sizeof(double) * nb * nl, cudaMemcpyDeviceToHost,
                       c->stream));
  std::vector<int> steps(nb);
  CK(cudaMemcpyAsync(steps.data(), c->steps_d.p, sizeof(int) * nb, cudaMemcpyDeviceToHost,
                     c->stream));
  int flags[4] = {0, 0, 0, 0};
  CK(cudaMemcpyAsync(flags, c->flags_d.p, sizeof(flags), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (flags[2]) return fail(c, RPA_ETIMEOUT, "a bounded tensor-core wait expired");
  if (flags[0] & 1) note_soft(c, RPA_EBREAKDOWN, "a Lanczos scalar (alpha or beta) is not finite");
  if (out.steps) std::memcpy(out.steps, steps.data(), sizeof(int) * nb);
  if (st) {
    CKS(timing_add(c, st, 5, 6, 5));
    for (int b = 0; b < nb; ++b) st->lanczos_steps_max = std::max(st->lanczos_steps_max, steps[b]);
    st->probe_points += nb;
  }
  return RPA_OK;
}

static void drop_lanes(rpa_ctx* c) {
  for (rpa_ctx* h : c->lanes) rpa_destroy(h);
  c->lanes.clear();
}

// Run count probe-points in waves; d/alpha/beta/steps are host arrays in input order.
// Blocks of the block Lanczos quadrature: runs of consecutive entries with one frequency and
// distinct points, at most bmax long, formed greedily from the first entry (single entries
// when bmax = 1).  Returns the start of every block and, last, count.
static std::vector<long long> lanczos_blocks(long long count, const long long* probe,
                                             const double* omg, int bmax) {
  std::vector<long long> bstart;
  for (long long i = 0; i < count;) {
    long long j = i + 1;
    while (j < count && j - i < bmax && omg[j] == omg[i]) {
      bool dup = false;
      for (long long q = i; q < j; ++q) dup = dup || probe[q] == probe[j];
      if (dup) break;
      ++j;
    }
    bstart.push_back(i);
    i = j;
  }
  bstart.push_back(count);
  return bstart;
}

static rpa_status run_probes(rpa_ctx* c, long long count, const long long* probe,
                             const double* omg, double* d, double* alpha, double* beta,
                             int* steps, rpa_stats* st) {
  if (count == 0) return RPA_OK;
  const int nb_max = choose_batch(c, count);
  CKS(ensure_workspace(c, nb_max));
  const int nl = c->opt.lanczos_max;
  const int bmax = c->opt.lanczos_block;
  if (bmax > 1) {
    // waves hold whole blocks
    const std::vector<long long> bstart = lanczos_blocks(count, probe, omg, bmax);
    const int wave_cap = std::max(nb_max, bmax);
    size_t bi = 0;
    while (bi + 1 < bstart.size()) {
      const long long s0 = bstart[bi];
      size_t be = bi + 1;
      while (be + 1 < bstart.size() && bstart[be + 1] - s0 <= wave_cap) ++be;
      const int nb = (int)(bstart[be] - s0);
      BlockLayout L;
      L.first.resize(nb);
      L.size.resize(nb);
      for (size_t q = bi; q < be; ++q) {
        const int f = (int)(bstart[q] - s0), n = (int)(bstart[q + 1] - bstart[q]);
        L.start.push_back(f);
        L.sz.push_back(n);
        for (int l = 0; l < n; ++l) {
          L.first[f + l] = f;
          L.size[f + l] = n;
        }
      }
      if (nb > nb_max) CKS(ensure_workspace(c, nb));
      WaveOut o;
      o.d = d + s0;
      o.alpha = nullptr;  // no scalar tridiagonal in block mode
      o.beta = nullptr;
      o.steps = steps ? steps + s0 : nullptr;
      if (alpha) std::memset(alpha + s0 * nl, 0, sizeof(double) * nb * nl);
      if (beta) std::memset(beta + s0 * nl, 0, sizeof(double) * nb * nl);
      CKS(run_wave(c, nb, probe + s0, omg + s0, o, st, &L));
      bi = be;
    }
    return RPA_OK;
  }
  for (long long s0 = 0; s0 < count; s0 += nb_max) {
    const int nb = (int)std::min<long long>(nb_max, count - s0);
    WaveOut o;
    o.d = d + s0;
    o.alpha = alpha ? alpha + s0 * nl : nullptr;
    o.beta = beta ? beta + s0 * nl : nullptr;
    o.steps = steps ? steps + s0 : nullptr;
    CKS(run_wave(c, nb, probe + s0, omg + s0, o, st));
  }
  return RPA_OK;
}

// helper contexts for options.lanes, set up from c's inputs (device copies on their own
// streams; the 1-D eigenbases are recomputed by each helper)
static rpa_status ensure_lanes(rpa_ctx* c, int k) {
  if ((int)c->lanes.size() >= k - 1) return RPA_OK;
  drop_lanes(c);
  CK(cudaStreamSynchronize(c->stream));
  for (int i = 0; i < k - 1; ++i) {
    rpa_ctx* h = nullptr;
    rpa_status st = rpa_create(&h, &c->grid, nullptr);
    if (st != RPA_OK) return fail(c, st, "creating a lane context failed");
    c->lanes.push_back(h);
    rpa_options o = c->opt;
    o.lanes = 1;
    if (st == RPA_OK) st = rpa_set_potential(h, c->d64.vloc.as<double>(), RPA_DEVICE);
    if (st == RPA_OK)
      st = rpa_set_projectors(h, c->hp_ng, c->hp_nnz.data(), c->hp_nproj.data(),
                              c->hp_idx.data(), c->hp_chi.data(), c->hp_gamma.data());
    if (st == RPA_OK)
      st = rpa_set_occupied(h, c->ns, c->d64.psi.as<double>(), c->eps_d.as<double>(),
                            RPA_DEVICE);
    if (st == RPA_OK) st = rpa_set_frequencies(h, c->nw, c->omega.data(), c->weight.data());
    if (st == RPA_OK) st = rpa_set_options(h, &o);
    if (st != RPA_OK) {
      const std::string m = h->err;
      drop_lanes(c);
      return fail(c, st, "setting up a lane context failed: " + m);
    }
    std::memcpy(h->tuned_ty, c->tuned_ty, sizeof(c->tuned_ty));
  }
  return RPA_OK;
}

static void add_stats(rpa_stats* a, const rpa_stats& b) {
  for (int i = 0; i < 8; ++i) {
    a->seconds_phase[i] += b.seconds_phase[i];
    a->kernel_seconds[i] += b.kernel_seconds[i];
    a->kernel_launches[i] += b.kernel_launches[i];
    a->kernel_bytes[i] += b.kernel_bytes[i];
  }
  a->probe_points += b.probe_points;
  a->matvecs += b.matvecs;
  a->solves += b.solves;
  a->cocg_iters += b.cocg_iters;
  a->refine_rounds += b.refine_rounds;
  a->nonconv_solves += b.nonconv_solves;
  a->breakdown_solves += b.breakdown_solves;
  a->max_cocg_iters = std::max(a->max_cocg_iters, b.max_cocg_iters);
  a->lanczos_steps_max = std::max(a->lanczos_steps_max, b.lanczos_steps_max);
  if (!a->precision_bytes) a->precision_bytes = b.precision_bytes;
}

// options.lanes = k > 1 (scalar Lanczos only): the probe-points are dealt round-robin to k
// lanes -- this context and k - 1 helpers, each with its own stream and workspace and each
// sizing its waves from 1/k of the free memory -- run concurrently from k host threads, so
// that the COCG tail of one lane (few systems left, small latency-bound launches) overlaps
// the other lanes' work.  Results return in input order; statistics are summed.
static rpa_status run_probes_lanes(rpa_ctx* c, long long count, const long long* probe,
                                   const double* omg, double* d, double* alpha, double* beta,
                                   int* steps, rpa_stats* st) {
  const int k = (int)std::min<long long>(c->opt.lanes, count);
  if (k <= 1 || c->opt.lanczos_block > 1)
    return run_probes(c, count, probe, omg, d, alpha, beta, steps, st);
  CKS(ensure_lanes(c, k));
  const int nl = c->opt.lanczos_max;
  struct Part {
    std::vector<long long> idx, pr;
    std::vector<double> om, d, al, be;
    std::vector<int> sp;
    rpa_stats stats;
    rpa_status rs = RPA_OK;
  };
  std::vector<Part> parts(k);
  for (long long i = 0; i < count; ++i) {
    Part& P = parts[i % k];
    P.idx.push_back(i);
    P.pr.push_back(probe[i]);
    P.om.push_back(omg[i]);
  }
  std::vector<rpa_ctx*> ctx(k);
  ctx[0] = c;
  for (int l = 1; l < k; ++l) ctx[l] = c->lanes[l - 1];
  for (int l = 0; l < k; ++l) {
    Part& P = parts[l];
    const size_t n = P.idx.size();
    P.d.assign(n, 0.0);
    if (alpha) P.al.assign(n * nl, 0.0);
    if (beta) P.be.assign(n * nl, 0.0);
    if (steps) P.sp.assign(n, 0);
    std::memset(&P.stats, 0, sizeof(P.stats));
    ctx[l]->mem_share = 1.0 / k;
    ctx[l]->soft = RPA_OK;
  }
  rpa_stats* parent_prof = c->prof_stats;
  std::vector<std::thread> th;
  for (int l = 0; l < k; ++l)
    th.emplace_back([&, l]() {
      Part& P = parts[l];
      rpa_ctx* h = ctx[l];
      cudaSetDevice(h->device);
      h->prof_stats = st ? &P.stats : nullptr;
      P.rs = run_probes(h, (long long)P.idx.size(), P.pr.data(), P.om.data(), P.d.data(),
                        alpha ? P.al.data() : nullptr, beta ? P.be.data() : nullptr,
                        steps ? P.sp.data() : nullptr, st ? &P.stats : nullptr);
      h->prof_stats = nullptr;
    });
  for (auto& t : th) t.join();
  c->prof_stats = parent_prof;
  for (int l = 0; l < k; ++l) ctx[l]->mem_share = 1.0;
  for (int l = 0; l < k; ++l) {
    if (parts[l].rs != RPA_OK) {
      const std::string m = ctx[l]->err;
      return l == 0 ? parts[0].rs : fail(c, parts[l].rs, "lane " + std::to_string(l) + ": " + m);
    }
  }
  for (int l = 1; l < k; ++l)
    if (ctx[l]->soft != RPA_OK) note_soft(c, ctx[l]->soft, ctx[l]->soft_msg.c_str());
  if (c->tuned_ty[0][0] == -1) std::memcpy(c->tuned_ty, ctx[1]->tuned_ty, sizeof(c->tuned_ty));
  for (int l = 0; l < k; ++l) {
    const Part& P = parts[l];
    for (size_t q = 0; q < P.idx.size(); ++q) {
      const long long i = P.idx[q];
      d[i] = P.d[q];
      if (alpha) std::memcpy(alpha + i * nl, P.al.data() + q * nl, sizeof(double) * nl);
      if (beta) std::memcpy(beta + i * nl, P.be.data() + q * nl, sizeof(double) * nl);
      if (steps) steps[i] = P.sp[q];
    }
    if (st) {
      add_stats(st, P.stats);
      if (l == 0) {
        st->tile_rows = P.stats.tile_rows;
        st->tile_rows_tail = P.stats.tile_rows_tail;
      }
    }
  }
  return RPA_OK;
}

// ---------------------------------------------------------------------------------------------
// interpolation (Section 3.2) and E_c
// ---------------------------------------------------------------------------------------------
static std::vector<long long> coarse_nodes(int n, int g, int bc) {
  std::vector<long long> v;
  for (int i = 0; i < n; i += g) v.push_back(i);
  if (bc == RPA_DIRICHLET && v.back() != n - 1) v.push_back(n - 1);
  return v;
}

static rpa_status build_interp(rpa_ctx* c) {
  const int kind = c->opt.interp;
  bool same = c->interp_built == kind;
  for (int a = 0; a < 3; ++a) same = same && c->stride_built[a] == c->opt.stride[a];
  if (same) return RPA_OK;
  for (int a = 0; a < 3; ++a) {
    const int n = c->grid.n[a], g = c->opt.stride[a];
    c->cnodes[a] = coarse_nodes(n, g, c->grid.bc[a]);
    const int m = (int)c->cnodes[a].size();
    int k = kind;
    if (g == 1) k = RPA_INTERP_NONE;
    if (k == RPA_INTERP_FOURIER && (c->grid.bc[a] != RPA_PERIODIC || n % g != 0))
      return fail(c, RPA_EINVAL, "Fourier interpolation needs periodic axes with n divisible by g");
    if (k == RPA_INTERP_TRICUBIC && c->grid.bc[a] == RPA_PERIODIC && m > 1 && m < 4)
      return fail(c, RPA_EINVAL, "tricubic interpolation on a periodic axis needs >= 4 coarse nodes");
    if (k == RPA_INTERP_TRILINEAR && c->grid.bc[a] == RPA_PERIODIC && m > 1 && m < 2)
      return fail(c, RPA_EINVAL, "trilinear interpolation needs >= 2 coarse nodes");
    if (k == RPA_INTERP_NONE && g != 1)
      return fail(c, RPA_EINVAL, "interp NONE requires stride 1");
    CK(c->cnodes_d[a].ensure(sizeof(long long) * m));
    CK(cudaMemcpyAsync(c->cnodes_d[a].p, c->cnodes[a].data(), sizeof(long long) * m,
                       cudaMemcpyHostToDevice, c->stream));
    CK(c->interpWt[a].ensure(sizeof(double) * (size_t)m * n));
    CK(interp_matrix(n, m, c->grid.bc[a], k, c->cnodes_d[a].as<long long>(),
                     c->interpWt[a].as<double>(), c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  c->interp_built = kind;
  for (int a = 0; a < 3; ++a) c->stride_built[a] = c->opt.stride[a];
  return RPA_OK;
}

static long long num_probes(rpa_ctx* c) {
  long long P = 1;
  for (int a = 0; a < 3; ++a) P *= (long long)coarse_nodes(c->grid.n[a], c->opt.stride[a], c->grid.bc[a]).size();
  return P;
}

// d_coarse (device, nw x P) -> d_fine (device, nw x N_d) and E_c (device scalar)
static rpa_status interpolate_dev(rpa_ctx* c, const double* dco, double* dfi, double* ec_dev) {
  CKS(build_interp(c));
  const int m[3] = {(int)c->cnodes[0].size(), (int)c->cnodes[1].size(), (int)c->cnodes[2].size()};
  const int* n = c->grid.n;
  const long long P = (long long)m[0] * m[1] * m[2];
  DevBuf t1, t2, part;
  CK(t1.ensure(sizeof(double) * c->nw * (long long)n[0] * m[1] * m[2]));
  CK(t2.ensure(sizeof(double) * c->nw * (long long)n[0] * n[1] * m[2]));
  int d0[3] = {m[0], m[1], m[2]};
  CK((mode_product<double, double, double>(dco, P, t1.as<double>(), (long long)n[0] * m[1] * m[2],
                                           c->interpWt[0].as<double>(), 0, d0, n[0], c->nw,
                                           nullptr, c->stream)));
  int d1[3] = {n[0], m[1], m[2]};
  CK((mode_product<double, double, double>(t1.as<double>(), (long long)n[0] * m[1] * m[2],
                                           t2.as<double>(), (long long)n[0] * n[1] * m[2],
                                           c->interpWt[1].as<double>(), 1, d1, n[1], c->nw,
                                           nullptr, c->stream)));
  int d2[3] = {n[0], n[1], m[2]};
  CK((mode_product<double, double, double>(t2.as<double>(), (long long)n[0] * n[1] * m[2], dfi,
                                           c->nd, c->interpWt[2].as<double>(), 2, d2, n[2],
                                           c->nw, nullptr, c->stream)));
  const int nblk = (int)std::max<long long>(1, std::min<long long>(256, (c->nd + 1023) / 1024));
  CK(part.ensure(sizeof(double) * nblk * c->nw));
  CK(ec_reduce(c->nd, c->nw, dfi, c->weight_d.as<double>(), part.as<double>(), nblk, ec_dev,
               c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return RPA_OK;
}

// ---------------------------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------------------------
static rpa_status check_ready(rpa_ctx* c, bool need_freq) {
  if (!c) return RPA_EINVAL;
  if (!c->have_vloc) return fail(c, RPA_ESTATE, "rpa_set_potential has not been called");
  if (!c->have_occ) return fail(c, RPA_ESTATE, "rpa_set_occupied has not been called");
  if (need_freq && !c->have_freq) return fail(c, RPA_ESTATE, "no frequencies set");
  CK(cudaSetDevice(c->device));
  return RPA_OK;
}

extern "C" {

rpa_status rpa_default_options(rpa_options* o) {
  if (!o) return RPA_EINVAL;
  std::memset(o, 0, sizeof(*o));
  o->lanczos_max = 20;
  o->lanczos_rtol = 0.0;
  o->stern_tol = 1e-10;
  o->stern_maxit = 20000;
  o->precision = RPA_FP64;
  o->reorth = 1;
  o->stride[0] = o->stride[1] = o->stride[2] = 1;
  o->interp = RPA_INTERP_TRICUBIC;
  o->batch = 0;
  o->fkind = RPA_F_LOG;
  o->refine = 4;
  o->inner_tol = 0.0;
  o->tile = -1;
  o->graphs = 2;
  o->lanczos_block = 1;
  o->refine_restart = 0;
  o->debug_expire_waits = 0;
  o->lanes = 1;
  return RPA_OK;
}

rpa_status rpa_create(rpa_ctx** out, const rpa_grid* g, void* stream) {
  if (!out || !g) return RPA_EINVAL;
  *out = nullptr;
  long long nd = 1;
  for (int a = 0; a < 3; ++a) {
    if (g->n[a] < 1 || g->n[a] > 1024 || !(g->h[a] > 0.0) ||
        (g->bc[a] != RPA_PERIODIC && g->bc[a] != RPA_DIRICHLET))
      return RPA_EINVAL;
    nd *= g->n[a];
  }
  if (g->fd_radius < 1 || g->fd_radius > kMaxRadius || nd >= (1LL << 31)) return RPA_EINVAL;
  rpa_ctx* c = new (std::nothrow) rpa_ctx();
  if (!c) return RPA_ENOMEM;
  c->grid = *g;
  c->nd = nd;
  c->dV = g->h[0] * g->h[1] * g->h[2];
  rpa_default_options(&c->opt);
  if (cudaGetDevice(&c->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
    delete c;
    return RPA_ECUDA;
  }
  if (stream) {
    c->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return RPA_ECUDA;
    }
    c->own_stream = true;
  }
  if (cudaMallocHost(&c->pinned, 64 * sizeof(int)) != cudaSuccess) {
    rpa_destroy(c);
    return RPA_ENOMEM;
  }
  c->have_events = true;
  for (int i = 0; i < 8; ++i)
    if (cudaEventCreate(&c->ev[i]) != cudaSuccess) c->have_events = false;
  c->have_pev = true;
  for (int i = 0; i < 4 * 7; ++i)
    if (cudaEventCreate(&c->pev[i]) != cudaSuccess) c->have_pev = false;
  make_stencil<double>(c->grid, c->d64.st);
  make_stencil<float>(c->grid, c->d32.st);
  // empty nonlocal part
  std::vector<int> zoff(nd + 1, 0);
  rpa_status st = RPA_OK;
  if (c->p_off.ensure(sizeof(int) * (nd + 1)) != cudaSuccess ||
      cudaMemcpy(c->p_off.p, zoff.data(), sizeof(int) * (nd + 1), cudaMemcpyHostToDevice) !=
          cudaSuccess)
    st = RPA_ECUDA;
  if (st == RPA_OK) st = build_nu(c);
  if (st != RPA_OK) {
    rpa_destroy(c);
    return st;
  }
  *out = c;
  return RPA_OK;
}

void rpa_destroy(rpa_ctx* c) {
  if (!c) return;
  drop_lanes(c);
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->have_events)
    for (int i = 0; i < 8; ++i) cudaEventDestroy(c->ev[i]);
  if (c->have_pev)
    for (int i = 0; i < 4 * 7; ++i) cudaEventDestroy(c->pev[i]);
  for (auto& g : c->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  if (c->pinned) cudaFreeHost(c->pinned);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

rpa_status rpa_set_potential(rpa_ctx* c, const double* vloc, int where) {
  if (!c || !vloc) return RPA_EINVAL;
  CK(cudaSetDevice(c->device));
  CK(c->d64.vloc.ensure(sizeof(double) * c->nd));
  CK(c->d32.vloc.ensure(sizeof(float) * c->nd));
  CKS(copy_in(c, c->d64.vloc.p, vloc, sizeof(double) * c->nd, where));
  CK(convert_d2f(c->d64.vloc.as<double>(), c->d32.vloc.as<float>(), c->nd, c->stream));
  CK(c->vloc2.ensure(sizeof(float2) * c->nd));
  CK(convert_d2df(c->d64.vloc.as<double>(), c->vloc2.as<float2>(), c->nd, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->have_vloc = true;
  drop_lanes(c);
  return RPA_OK;
}

rpa_status rpa_set_projectors(rpa_ctx* c, int ngroups, const int* nnz, const int* nproj,
                              const int* idx, const double* chi, const double* gamma) {
  if (!c || ngroups < 0) return RPA_EINVAL;
  CK(cudaSetDevice(c->device));
  const long long nd = c->nd;
  // split groups into internal groups of <= 4 projectors sharing the support
  std::vector<int> goff(1, 0), gidx;
  std::vector<double> gchi, gcoef;
  std::vector<std::vector<std::pair<int, long long>>> at;  // unused placeholder
  long long ioff = 0, coff = 0, goff_in = 0;
  for (int g = 0; g < ngroups; ++g) {
    if (!nnz || !nproj || !idx || !chi || !gamma) return fail(c, RPA_EINVAL, "null projector array");
    const int z = nnz[g], np = nproj[g];
    if (z < 0 || np < 1 || np > 16) return fail(c, RPA_EINVAL, "projector group size out of range");
    for (int e = 0; e < z; ++e)
      if (idx[ioff + e] < 0 || idx[ioff + e] >= nd)
        return fail(c, RPA_EINVAL, "projector index out of range");
    std::vector<int> order(z);
    for (int e = 0; e < z; ++e) order[e] = e;
    std::sort(order.begin(), order.end(),
              [&](int a, int b) { return idx[ioff + a] < idx[ioff + b]; });
    for (int e = 0; e + 1 < z; ++e)
      if (idx[ioff + order[e]] == idx[ioff + order[e + 1]])
        return fail(c, RPA_EINVAL, "duplicate grid index within a projector group");
    for (int l0 = 0; l0 < np; l0 += kProjChunk) {
      for (int oe = 0; oe < z; ++oe) {
        const int e = order[oe];
        gidx.push_back(idx[ioff + e]);
        for (int l = 0; l < kProjChunk; ++l)
          gchi.push_back(l0 + l < np ? chi[coff + (long long)(l0 + l) * z + e] : 0.0);
      }
      for (int l = 0; l < kProjChunk; ++l)
        gcoef.push_back(l0 + l < np ? gamma[goff_in + l0 + l] * c->dV : 0.0);
      goff.push_back((int)gidx.size());
    }
    ioff += z;
    coff += (long long)np * z;
    goff_in += np;
  }
  const int NG = (int)goff.size() - 1;
  const long long E = (long long)gidx.size();
  if (E >= (1LL << 31)) return fail(c, RPA_EINVAL, "too many projector entries");
  // point-major copy
  std::vector<int> poff(nd + 1, 0);
  for (long long e = 0; e < E; ++e) poff[gidx[e] + 1]++;
  for (long long p = 0; p < nd; ++p) poff[p + 1] += poff[p];
  std::vector<int> pgrp(std::max<long long>(E, 1)), fill(poff.begin(), poff.end() - 1);
  std::vector<double> pchi(std::max<long long>(E, 1) * kProjChunk);
  for (int g = 0; g < NG; ++g)
    for (int e = goff[g]; e < goff[g + 1]; ++e) {
      const int pt = gidx[e];
      const int slot = fill[pt]++;
      pgrp[slot] = g;
      for (int l = 0; l < kProjChunk; ++l) pchi[(size_t)slot * kProjChunk + l] = gchi[(size_t)e * kProjChunk + l];
    }
  // projector overlaps of groups with common support (point-major: every pair of entries at
  // a point), as 4 x 4 blocks per (group, group) pair, rows by group
  std::vector<int> soff(NG + 1, 0), snbr;
  std::vector<double> sblk;
  {
    std::vector<std::vector<std::pair<int, std::array<double, 16>>>> rows(NG);
    for (long long q = 0; q < nd; ++q)
      for (int e1 = poff[q]; e1 < poff[q + 1]; ++e1)
        for (int e2 = poff[q]; e2 < poff[q + 1]; ++e2) {
          auto& row = rows[pgrp[e1]];
          const int h = pgrp[e2];
          size_t k = 0;
          while (k < row.size() && row[k].first != h) ++k;
          if (k == row.size()) {
            row.emplace_back(h, std::array<double, 16>{});
          }
          for (int l = 0; l < kProjChunk; ++l)
            for (int m = 0; m < kProjChunk; ++m)
              row[k].second[l * 4 + m] += pchi[(size_t)e1 * kProjChunk + l] *
                                          pchi[(size_t)e2 * kProjChunk + m];
        }
    for (int g = 0; g < NG; ++g) {
      std::sort(rows[g].begin(), rows[g].end(),
                [](const auto& a, const auto& b) { return a.first < b.first; });
      for (const auto& nb : rows[g]) {
        snbr.push_back(nb.first);
        sblk.insert(sblk.end(), nb.second.begin(), nb.second.end());
      }
      soff[g + 1] = (int)snbr.size();
    }
  }
  {
    const size_t nb = std::max<size_t>(snbr.size(), 1);
    std::vector<float> sblk_f(sblk.begin(), sblk.end());
    CK(c->s_off.ensure(sizeof(int) * soff.size()));
    CK(c->s_nbr.ensure(sizeof(int) * nb));
    CK(c->d64.s_blk.ensure(sizeof(double) * nb * 16));
    CK(c->d32.s_blk.ensure(sizeof(float) * nb * 16));
    CK(cudaMemcpy(c->s_off.p, soff.data(), sizeof(int) * soff.size(), cudaMemcpyHostToDevice));
    if (!snbr.empty()) {
      CK(cudaMemcpy(c->s_nbr.p, snbr.data(), sizeof(int) * snbr.size(), cudaMemcpyHostToDevice));
      CK(cudaMemcpy(c->d64.s_blk.p, sblk.data(), sizeof(double) * sblk.size(),
                    cudaMemcpyHostToDevice));
      CK(cudaMemcpy(c->d32.s_blk.p, sblk_f.data(), sizeof(float) * sblk_f.size(),
                    cudaMemcpyHostToDevice));
    }
  }
  // per 1-D COCG tile (kTile consecutive points): for every group with entries in the tile,
  // the contiguous range of its (index-sorted) group-major entries that falls in the tile
  const long long ntile = (nd + kTile - 1) / kTile;
  std::vector<int> troff(ntile + 1, 0), trng;
  {
    std::vector<std::vector<int>> per(ntile);
    for (int g = 0; g < NG; ++g) {
      int e = goff[g];
      while (e < goff[g + 1]) {
        const long long t = gidx[e] / kTile;
        int f = e;
        while (f < goff[g + 1] && gidx[f] / kTile == t) ++f;
        per[t].push_back(g);
        per[t].push_back(e);
        per[t].push_back(f);
        e = f;
      }
    }
    for (long long t = 0; t < ntile; ++t) {
      troff[t + 1] = troff[t] + (int)(per[t].size() / 3);
      trng.insert(trng.end(), per[t].begin(), per[t].end());
    }
  }
  if (trng.empty()) trng.assign(3, 0);
  CK(c->tile_roff.ensure(sizeof(int) * troff.size()));
  CK(c->tile_ranges.ensure(sizeof(int) * trng.size()));
  CK(cudaMemcpy(c->tile_roff.p, troff.data(), sizeof(int) * troff.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(c->tile_ranges.p, trng.data(), sizeof(int) * trng.size(), cudaMemcpyHostToDevice));
  std::vector<float> gchi_f(gchi.begin(), gchi.end()), gcoef_f(gcoef.begin(), gcoef.end()),
      pchi_f(pchi.begin(), pchi.end());
  // lo parts of the double-float pairs (hi = the FP32 copy)
  auto lo_of = [](const std::vector<double>& v, const std::vector<float>& h) {
    std::vector<float> lo(v.size());
    for (size_t i = 0; i < v.size(); ++i) lo[i] = (float)(v[i] - (double)h[i]);
    return lo;
  };
  const std::vector<float> gchi_lo = lo_of(gchi, gchi_f), pchi_lo = lo_of(pchi, pchi_f),
                           gcoef_lo = lo_of(gcoef, gcoef_f);
  const size_t Eb = std::max<long long>(E, 1);
  CK(c->g_off.ensure(sizeof(int) * goff.size()));
  CK(c->g_idx.ensure(sizeof(int) * Eb));
  CK(c->p_off.ensure(sizeof(int) * (nd + 1)));
  CK(c->p_grp.ensure(sizeof(int) * Eb));
  CK(c->d64.g_chi.ensure(sizeof(double) * Eb * kProjChunk));
  CK(c->d32.g_chi.ensure(sizeof(float) * Eb * kProjChunk));
  CK(c->d64.p_chi.ensure(sizeof(double) * Eb * kProjChunk));
  CK(c->d32.p_chi.ensure(sizeof(float) * Eb * kProjChunk));
  CK(c->d64.coef.ensure(sizeof(double) * std::max(NG, 1) * kProjChunk));
  CK(c->d32.coef.ensure(sizeof(float) * std::max(NG, 1) * kProjChunk));
  CK(c->g_chi_lo.ensure(sizeof(float) * Eb * kProjChunk));
  CK(c->p_chi_lo.ensure(sizeof(float) * Eb * kProjChunk));
  CK(c->coef_lo.ensure(sizeof(float) * std::max(NG, 1) * kProjChunk));
  CK(cudaMemcpy(c->g_off.p, goff.data(), sizeof(int) * goff.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(c->p_off.p, poff.data(), sizeof(int) * (nd + 1), cudaMemcpyHostToDevice));
  if (E > 0) {
    CK(cudaMemcpy(c->g_idx.p, gidx.data(), sizeof(int) * E, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->p_grp.p, pgrp.data(), sizeof(int) * E, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->d64.g_chi.p, gchi.data(), sizeof(double) * E * kProjChunk, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->d32.g_chi.p, gchi_f.data(), sizeof(float) * E * kProjChunk, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->d64.p_chi.p, pchi.data(), sizeof(double) * E * kProjChunk, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->d32.p_chi.p, pchi_f.data(), sizeof(float) * E * kProjChunk, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->d64.coef.p, gcoef.data(), sizeof(double) * NG * kProjChunk, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->d32.coef.p, gcoef_f.data(), sizeof(float) * NG * kProjChunk, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->g_chi_lo.p, gchi_lo.data(), sizeof(float) * E * kProjChunk, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->p_chi_lo.p, pchi_lo.data(), sizeof(float) * E * kProjChunk, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->coef_lo.p, gcoef_lo.data(), sizeof(float) * NG * kProjChunk, cudaMemcpyHostToDevice));
  }
  c->ngroup = NG;
  // host copy of the inputs, for lane contexts
  long long nidx = 0, nchi = 0, ngam = 0;
  for (int g = 0; g < ngroups; ++g) {
    nidx += nnz[g];
    nchi += (long long)nproj[g] * nnz[g];
    ngam += nproj[g];
  }
  c->hp_ng = ngroups;
  c->hp_nnz.assign(nnz, nnz + ngroups);
  c->hp_nproj.assign(nproj, nproj + ngroups);
  c->hp_idx.assign(idx, idx + nidx);
  c->hp_chi.assign(chi, chi + nchi);
  c->hp_gamma.assign(gamma, gamma + ngam);
  drop_lanes(c);
  return RPA_OK;
}

rpa_status rpa_set_occupied(rpa_ctx* c, int ns, const double* psi, const double* eps, int where) {
  if (!c || !psi || !eps || ns < 1 || ns > 1024) return RPA_EINVAL;
  CK(cudaSetDevice(c->device));
  std::vector<double> e(ns);
  if (where == RPA_DEVICE) {
    CK(cudaMemcpyAsync(e.data(), eps, sizeof(double) * ns, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  } else
    std::memcpy(e.data(), eps, sizeof(double) * ns);
  for (int i = 0; i + 1 < ns; ++i)
    if (!(e[i] <= e[i + 1])) return fail(c, RPA_ENOGAP, "eps must be ascending");
  const long long n = (long long)ns * c->nd;
  CK(c->d64.psi.ensure(sizeof(double) * n));
  CK(c->d32.psi.ensure(sizeof(float) * n));
  CK(c->eps_d.ensure(sizeof(double) * ns));
  CKS(copy_in(c, c->d64.psi.p, psi, sizeof(double) * n, where));
  CK(convert_d2f(c->d64.psi.as<double>(), c->d32.psi.as<float>(), n, c->stream));
  CK(c->psi2.ensure(sizeof(float2) * n));
  CK(convert_d2df(c->d64.psi.as<double>(), c->psi2.as<float2>(), n, c->stream));
  CK(cudaMemcpyAsync(c->eps_d.p, e.data(), sizeof(double) * ns, cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->eps_h = e;
  c->ns = ns;
  c->have_occ = true;
  c->ws_nb = 0;
  drop_lanes(c);
  return RPA_OK;
}

rpa_status rpa_set_frequencies(rpa_ctx* c, int nw, const double* omega, const double* weight) {
  if (!c || nw < 1 || nw > 64 || !omega || !weight) return RPA_EINVAL;
  for (int k = 0; k < nw; ++k)
    if (!(omega[k] > 0.0) || !std::isfinite(weight[k]))
      return fail(c, RPA_EINVAL, "frequencies must be positive and weights finite");
  CK(cudaSetDevice(c->device));
  c->omega.assign(omega, omega + nw);
  c->weight.assign(weight, weight + nw);
  CK(c->omega_d.ensure(sizeof(double) * nw));
  CK(c->weight_d.ensure(sizeof(double) * nw));
  CK(cudaMemcpy(c->omega_d.p, omega, sizeof(double) * nw, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(c->weight_d.p, weight, sizeof(double) * nw, cudaMemcpyHostToDevice));
  c->nw = nw;
  c->have_freq = true;
  drop_lanes(c);
  return RPA_OK;
}

rpa_status rpa_gl_frequencies(int nw, double* omega, double* weight) {
  if (nw < 1 || nw > 64 || !omega || !weight) return RPA_EINVAL;
  double* d = nullptr;
  if (cudaMalloc(&d, sizeof(double) * 2 * nw) != cudaSuccess) return RPA_ENOMEM;
  rpa_status st = RPA_OK;
  if (gl_nodes(nw, d, d + nw, 0) != cudaSuccess ||
      cudaMemcpy(omega, d, sizeof(double) * nw, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(weight, d + nw, sizeof(double) * nw, cudaMemcpyDeviceToHost) != cudaSuccess)
    st = RPA_ECUDA;
  cudaFree(d);
  return st;
}

rpa_status rpa_set_options(rpa_ctx* c, const rpa_options* o) {
  if (!c || !o) return RPA_EINVAL;
  if (o->lanczos_max < 1 || o->lanczos_max > kMaxLanczos) return fail(c, RPA_EINVAL, "lanczos_max out of range");
  if (!(o->stern_tol > 0.0) || o->stern_maxit < 1) return fail(c, RPA_EINVAL, "bad Sternheimer tolerance");
  if (o->precision != RPA_FP64 && o->precision != RPA_MIXED && o->precision != RPA_MIXED_BF16)
    return fail(c, RPA_EINVAL, "bad precision");
  if (o->interp < RPA_INTERP_NONE || o->interp > RPA_INTERP_FOURIER) return fail(c, RPA_EINVAL, "bad interp");
  if (o->fkind < RPA_F_LOG || o->fkind > RPA_F_X2) return fail(c, RPA_EINVAL, "bad fkind");
  if (o->lanczos_rtol < 0.0 || o->refine < 0 || o->refine > 20 || o->batch < 0)
    return fail(c, RPA_EINVAL, "bad option");
  for (int a = 0; a < 3; ++a)
    if (o->stride[a] < 1 || o->stride[a] > c->grid.n[a]) return fail(c, RPA_EINVAL, "bad stride");
  if (o->tile == kTileX2Packed) {
    if (o->precision == RPA_FP64 || !x2p_tile_fits(c->grid.n[0], c->grid.fd_radius))
      return fail(c, RPA_EINVAL, "packed-row two-point tiles need the mixed form, an even nx "
                                 "from 26 to 64 and stencil radius 6");
  } else if (is_x2(o->tile)) {
    if (o->precision == RPA_FP64 || !x2_tile_fits(c->grid.n[0], c->grid.fd_radius))
      return fail(c, RPA_EINVAL, "two-point tiles need the mixed form and an even nx");
  } else if (is_band(o->tile)) {
    if (o->precision == RPA_FP64 ||
        !band_tile_fits(c->grid.n[0], c->grid.n[1], c->grid.fd_radius, band_rows(o->tile),
                        c->ngroup))
      return fail(c, RPA_EINVAL, "band tiles need the mixed form, an even nx <= 64 and a band "
                                 "height that divides ny");
  } else if (o->tile > 0) {
    const bool ok = o->precision == RPA_FP64
                        ? row_tile_fits<double>(c->grid.n[0], c->grid.n[1], c->grid.fd_radius, o->tile)
                        : row_tile_fits<float>(c->grid.n[0], c->grid.n[1], c->grid.fd_radius, o->tile);
    if (!ok) return fail(c, RPA_EINVAL, "row-tile height does not fit this grid");
  } else if (o->tile < -2) {  // -5 .. -100
    return fail(c, RPA_EINVAL, "bad tile option");
  }
  if (o->graphs < 0 || o->graphs > 2) return fail(c, RPA_EINVAL, "bad graphs option");
  if (o->lanes < 1 || o->lanes > 8) return fail(c, RPA_EINVAL, "lanes out of range");
  if (o->refine_restart != 0 && o->refine_restart != 1)
    return fail(c, RPA_EINVAL, "bad refine_restart option");
  if (o->debug_expire_waits != 0 && o->debug_expire_waits != 1)
    return fail(c, RPA_EINVAL, "bad debug_expire_waits option");
  if (o->lanczos_block < 1 || o->lanczos_block > block_max())
    return fail(c, RPA_EINVAL, "lanczos_block out of range");
  if (o->lanczos_block > 1 && (o->lanczos_rtol != 0.0 || !o->reorth))
    return fail(c, RPA_EINVAL, "block Lanczos needs full reorthogonalisation and no early exit");
  const bool realloc = o->precision != c->opt.precision || o->lanczos_max != c->opt.lanczos_max ||
                       o->refine != c->opt.refine;
  c->opt = *o;
  drop_lanes(c);
  if (realloc) c->ws_nb = 0;
  return RPA_OK;
}

rpa_status rpa_num_probes(rpa_ctx* c, long long* P) {
  if (!c || !P) return RPA_EINVAL;
  *P = num_probes(c);
  return RPA_OK;
}

rpa_status rpa_probe_indices(rpa_ctx* c, long long* idx) {
  if (!c || !idx) return RPA_EINVAL;
  std::vector<long long> cn[3];
  for (int a = 0; a < 3; ++a) cn[a] = coarse_nodes(c->grid.n[a], c->opt.stride[a], c->grid.bc[a]);
  long long q = 0;
  for (long long kz : cn[2])
    for (long long ky : cn[1])
      for (long long kx : cn[0]) idx[q++] = kx + (long long)c->grid.n[0] * (ky + (long long)c->grid.n[1] * kz);
  return RPA_OK;
}

rpa_status rpa_probe_density(rpa_ctx* c, int count, const long long* probe, const int* freq,
                             double* d, double* alpha, double* beta, int* steps, rpa_stats* st,
                             int where) {
  CKS(check_ready(c, true));
  if (count < 0 || (count > 0 && (!probe || !freq || !d))) return fail(c, RPA_EINVAL, "bad arguments");
  auto t0 = std::chrono::steady_clock::now();
  std::vector<long long> pr(count);
  std::vector<int> fq(count);
  if (where == RPA_DEVICE) {
    if (count > 0) {
      CK(cudaMemcpyAsync(pr.data(), probe, sizeof(long long) * count, cudaMemcpyDeviceToHost,
                         c->stream));
      CK(cudaMemcpyAsync(fq.data(), freq, sizeof(int) * count, cudaMemcpyDeviceToHost,
                         c->stream));
      CK(cudaStreamSynchronize(c->stream));
    }
  } else {
    std::memcpy(pr.data(), probe, sizeof(long long) * count);
    std::memcpy(fq.data(), freq, sizeof(int) * count);
  }
  std::vector<double> om(count);
  for (int i = 0; i < count; ++i) {
    if (pr[i] < 0 || pr[i] >= c->nd || fq[i] < 0 || fq[i] >= c->nw)
      return fail(c, RPA_EINVAL, "probe or frequency index out of range");
    om[i] = c->omega[fq[i]];
  }
  if (st) std::memset(st, 0, sizeof(*st));
  c->prof_stats = st;
  const int nl = c->opt.lanczos_max;
  std::vector<double> dh(count), ah(alpha ? (size_t)count * nl : 0), bh(beta ? (size_t)count * nl : 0);
  std::vector<int> sh(steps ? count : 0);
  c->soft = RPA_OK;
  rpa_status rs = run_probes_lanes(c, count, pr.data(), om.data(), dh.data(),
                                   alpha ? ah.data() : nullptr, beta ? bh.data() : nullptr,
                                   steps ? sh.data() : nullptr, st);
  c->prof_stats = nullptr;
  CKS(rs);
  CKS(copy_out(c, d, dh.data(), sizeof(double) * count, where));
  if (alpha) CKS(copy_out(c, alpha, ah.data(), sizeof(double) * count * nl, where));
  if (beta) CKS(copy_out(c, beta, bh.data(), sizeof(double) * count * nl, where));
  if (steps) CKS(copy_out(c, steps, sh.data(), sizeof(int) * count, where));
  CK(cudaStreamSynchronize(c->stream));
  if (st) st->seconds_total = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return soft_status(c);
}

rpa_status rpa_batch_energy(int nsys, rpa_ctx* const* sys, double* ec_out, rpa_stats* stats) {
  if (nsys < 0 || (nsys > 0 && (!sys || !ec_out))) return RPA_EINVAL;
  for (int i = 0; i < nsys; ++i) {
    if (!sys[i]) return RPA_EINVAL;
    for (int j = 0; j < i; ++j)
      if (sys[i] == sys[j]) return fail(sys[i], RPA_EINVAL, "contexts must be distinct");
  }
  std::vector<rpa_status> st(nsys, RPA_OK);
  std::vector<std::thread> th;
  th.reserve(nsys);
  for (int i = 0; i < nsys; ++i)
    th.emplace_back([&, i]() {
      cudaSetDevice(sys[i]->device);
      st[i] = rpa_energy_density(sys[i], nullptr, nullptr, &ec_out[i],
                                 stats ? &stats[i] : nullptr, RPA_HOST);
    });
  for (auto& t : th) t.join();
  for (int i = 0; i < nsys; ++i)
    if (st[i] != RPA_OK) return st[i];
  return RPA_OK;
}

rpa_status rpa_interpolate(rpa_ctx* c, const double* d_coarse, double* d_fine, double* ec,
                           int where) {
  if (!c || !d_coarse) return RPA_EINVAL;
  if (!c->have_freq) return fail(c, RPA_ESTATE, "no frequencies set");
  CK(cudaSetDevice(c->device));
  const long long P = num_probes(c);
  DevBuf dco, dfi, ecd;
  CK(dco.ensure(sizeof(double) * c->nw * P));
  CK(dfi.ensure(sizeof(double) * c->nw * c->nd));
  CK(ecd.ensure(sizeof(double)));
  CKS(copy_in(c, dco.p, d_coarse, sizeof(double) * c->nw * P, where));
  CKS(interpolate_dev(c, dco.as<double>(), dfi.as<double>(), ecd.as<double>()));
  if (d_fine) CKS(copy_out(c, d_fine, dfi.p, sizeof(double) * c->nw * c->nd, where));
  if (ec) CKS(copy_out(c, ec, ecd.p, sizeof(double), where));
  CK(cudaStreamSynchronize(c->stream));
  return RPA_OK;
}

// Fingerprint of everything that fixes d on C_g: grid, inputs (V_loc, projectors, occupied
// states and eigenvalues), frequencies, the coarse set and the options that change d.
static rpa_status problem_key(rpa_ctx* c, const std::vector<long long>& idx,
                              unsigned long long* key) {
  unsigned long long h = kFnvBasis;
  auto mix = [&h](const void* p, size_t n) { h = fnv1a(h, p, n); };
  auto mixv = [&mix](const auto& v) {
    const long long n = (long long)v.size();
    mix(&n, sizeof(n));
    if (n) mix(v.data(), sizeof(v[0]) * v.size());
  };
  const rpa_grid& g = c->grid;
  mix(g.n, sizeof(g.n));
  mix(g.h, sizeof(g.h));
  mix(g.bc, sizeof(g.bc));
  mix(&g.fd_radius, sizeof(g.fd_radius));
  // device inputs hashed through a bounded host buffer
  auto mixdev = [&](const void* d, size_t bytes) -> cudaError_t {
    std::vector<unsigned char> hb(std::min<size_t>(bytes, (size_t)8 << 20));
    mix(&bytes, sizeof(bytes));
    for (size_t off = 0; off < bytes; off += hb.size()) {
      const size_t n = std::min(hb.size(), bytes - off);
      const cudaError_t e = cudaMemcpy(hb.data(), static_cast<const unsigned char*>(d) + off, n,
                                       cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return e;
      mix(hb.data(), n);
    }
    return cudaSuccess;
  };
  CK(mixdev(c->d64.vloc.p, sizeof(double) * c->nd));
  CK(mixdev(c->d64.psi.p, sizeof(double) * c->ns * c->nd));
  mixv(c->eps_h);
  mix(&c->hp_ng, sizeof(c->hp_ng));
  mixv(c->hp_nnz);
  mixv(c->hp_nproj);
  mixv(c->hp_idx);
  mixv(c->hp_chi);
  mixv(c->hp_gamma);
  mixv(c->omega);
  mixv(idx);
  const rpa_options& o = c->opt;
  const double dopt[] = {o.lanczos_rtol, o.stern_tol, o.inner_tol};
  const int iopt[] = {o.lanczos_max, o.stern_maxit, o.precision, o.reorth,  o.fkind,
                      o.refine,      o.lanczos_block, o.refine_restart};
  mix(dopt, sizeof(dopt));
  mix(iopt, sizeof(iopt));
  *key = h;
  return RPA_OK;
}

rpa_status rpa_set_checkpoint(rpa_ctx* c, const char* path) {
  if (!c) return RPA_EINVAL;
  c->ckpt_path = path ? path : "";
  return RPA_OK;
}

rpa_status rpa_energy_density(rpa_ctx* c, double* d_coarse, double* d_fine, double* ec,
                              rpa_stats* st, int where) {
  CKS(check_ready(c, true));
  auto t0 = std::chrono::steady_clock::now();
  if (st) std::memset(st, 0, sizeof(*st));
  const long long P = num_probes(c);
  std::vector<long long> idx(P);
  CKS(rpa_probe_indices(c, idx.data()));
  const long long count = P * c->nw;
  std::vector<long long> pr(count);
  std::vector<double> om(count), dh(count);
  for (int k = 0; k < c->nw; ++k)
    for (long long j = 0; j < P; ++j) {
      pr[k * P + j] = idx[j];
      om[k * P + j] = c->omega[k];
    }
  c->soft = RPA_OK;
  c->soft_msg.clear();
  if (c->ckpt_path.empty()) {
    c->prof_stats = st;
    rpa_status rs = run_probes_lanes(c, count, pr.data(), om.data(), dh.data(), nullptr,
                                     nullptr, nullptr, st);
    c->prof_stats = nullptr;
    CKS(rs);
  } else {
    // resume: entries in the checkpoint are taken from it; the others run in blocks of one
    // wave per lane, each block's entries appended to the file when the block completes
    unsigned long long key = 0;
    CKS(problem_key(c, idx, &key));
    Checkpoint ck;
    std::vector<CkptRecord> recs;
    std::string msg;
    if (ck.open(c->ckpt_path, key, count, &recs, &msg) != RPA_OK) return fail(c, RPA_EINVAL, msg);
    std::vector<char> done(count, 0);
    for (const CkptRecord& r : recs) {
      dh[r.entry] = r.d;
      done[r.entry] = 1;
      if (r.status == RPA_ENOCONV || r.status == RPA_EBREAKDOWN)
        note_soft(c, (rpa_status)r.status, "a solve of an entry resumed from the checkpoint");
    }
    // Work goes in whole quadrature blocks (block Lanczos: the blocks of the uninterrupted
    // run, so that a resumed entry shares its block with the same points; a block counts as
    // done only when all its entries are in the file, else it is recomputed whole).
    const std::vector<long long> qb =
        lanczos_blocks(count, pr.data(), om.data(), std::max(1, c->opt.lanczos_block));
    std::vector<long long> todo, todo_blk;  // undone entries; start of each undone block in todo
    for (size_t q = 0; q + 1 < qb.size(); ++q) {
      bool all = true;
      for (long long i = qb[q]; i < qb[q + 1]; ++i) all = all && done[i];
      if (all) continue;
      todo_blk.push_back((long long)todo.size());
      for (long long i = qb[q]; i < qb[q + 1]; ++i) todo.push_back(i);
    }
    todo_blk.push_back((long long)todo.size());
    const long long block =
        (long long)choose_batch(c, (long long)todo.size()) * std::max(1, c->opt.lanes);
    std::vector<long long> bpr;
    std::vector<double> bom, bd;
    for (size_t q0 = 0; q0 + 1 < todo_blk.size();) {
      // whole blocks up to `block` entries (at least one block)
      size_t q1 = q0 + 1;
      while (q1 + 1 < todo_blk.size() && todo_blk[q1 + 1] - todo_blk[q0] <= block) ++q1;
      const size_t b0 = (size_t)todo_blk[q0], n = (size_t)(todo_blk[q1] - todo_blk[q0]);
      q0 = q1;
      bpr.resize(n);
      bom.resize(n);
      bd.assign(n, 0.0);
      for (size_t i = 0; i < n; ++i) {
        bpr[i] = pr[todo[b0 + i]];
        bom[i] = om[todo[b0 + i]];
      }
      const rpa_status prev = c->soft;
      const std::string prev_msg = c->soft_msg;
      c->soft = RPA_OK;
      c->prof_stats = st;
      rpa_status rs = run_probes_lanes(c, (long long)n, bpr.data(), bom.data(), bd.data(),
                                       nullptr, nullptr, nullptr, st);
      c->prof_stats = nullptr;
      const rpa_status bs = c->soft;
      const std::string bmsg = c->soft_msg;
      c->soft = prev;
      c->soft_msg = prev_msg;
      if (bs != RPA_OK) note_soft(c, bs, bmsg.c_str());
      CKS(rs);
      recs.resize(n);
      for (size_t i = 0; i < n; ++i) {
        const long long e = todo[b0 + i];
        dh[e] = bd[i];
        recs[i] = CkptRecord{e, bd[i], (int)bs, 0u};
      }
      if (ck.append(recs, &msg) != RPA_OK) return fail(c, RPA_EINVAL, msg);
    }
  }
  auto t1 = std::chrono::steady_clock::now();
  DevBuf dco, dfi, ecd;
  CK(dco.ensure(sizeof(double) * count));
  CK(dfi.ensure(sizeof(double) * c->nw * c->nd));
  CK(ecd.ensure(sizeof(double)));
  CK(cudaMemcpyAsync(dco.p, dh.data(), sizeof(double) * count, cudaMemcpyHostToDevice, c->stream));
  CKS(interpolate_dev(c, dco.as<double>(), dfi.as<double>(), ecd.as<double>()));
  if (d_coarse) CKS(copy_out(c, d_coarse, dco.p, sizeof(double) * count, where));
  if (d_fine) CKS(copy_out(c, d_fine, dfi.p, sizeof(double) * c->nw * c->nd, where));
  if (ec) CKS(copy_out(c, ec, ecd.p, sizeof(double), where));
  CK(cudaStreamSynchronize(c->stream));
  auto t2 = std::chrono::steady_clock::now();
  if (st) {
    st->seconds_phase[6] += std::chrono::duration<double>(t2 - t1).count();
    st->seconds_total = std::chrono::duration<double>(t2 - t0).count();
  }
  return soft_status(c);
}

rpa_status rpa_apply_h(rpa_ctx* c, int count, const double* x, const double* sigma, double* y,
                       int where) {
  if (!c || count < 0 || (count > 0 && (!x || !sigma || !y))) return RPA_EINVAL;
  if (!c->have_vloc) return fail(c, RPA_ESTATE, "rpa_set_potential has not been called");
  if (count == 0) return RPA_OK;
  CK(cudaSetDevice(c->device));
  const long long n = (long long)count * c->nd;
  DevBuf xd, yd, sd, cd;
  CK(xd.ensure(sizeof(cpx<double>) * n));
  CK(yd.ensure(sizeof(cpx<double>) * n));
  CK(sd.ensure(sizeof(cpx<double>) * count));
  CK(cd.ensure(sizeof(cpx<double>) * count * std::max(1, c->ngroup) * kProjChunk));
  CKS(copy_in(c, xd.p, x, sizeof(cpx<double>) * n, where));
  CKS(copy_in(c, sd.p, sigma, sizeof(cpx<double>) * count, where));
  if (c->opt.precision == RPA_FP64) {
    CK(apply_h<double>(c->d64.st, c->d64.vloc.as<double>(), nlview<double>(c), c->nd, count,
                       xd.as<cpx<double>>(), sd.as<cpx<double>>(), cd.as<cpx<double>>(),
                       yd.as<cpx<double>>(), c->stream));
  } else {
    DevBuf xf, yf, sf;
    CK(xf.ensure(sizeof(cpx<float>) * n));
    CK(yf.ensure(sizeof(cpx<float>) * n));
    CK(sf.ensure(sizeof(cpx<float>) * count));
    CK(convert_d2f(xd.as<double>(), xf.as<float>(), 2 * n, c->stream));
    CK(convert_d2f(sd.as<double>(), sf.as<float>(), 2 * count, c->stream));
    CK(apply_h<float>(c->d32.st, c->d32.vloc.as<float>(), nlview<float>(c), c->nd, count,
                      xf.as<cpx<float>>(), sf.as<cpx<float>>(), cd.as<cpx<float>>(),
                      yf.as<cpx<float>>(), c->stream));
    CK(convert_f2d(yf.as<float>(), yd.as<double>(), 2 * n, c->stream));
  }
  CKS(copy_out(c, y, yd.p, sizeof(cpx<double>) * n, where));
  CK(cudaStreamSynchronize(c->stream));
  return RPA_OK;
}

rpa_status rpa_apply_nu_half(rpa_ctx* c, int count, const double* q, double* u, int where) {
  if (!c || count < 0 || (count > 0 && (!q || !u))) return RPA_EINVAL;
  if (count == 0) return RPA_OK;
  CK(cudaSetDevice(c->device));
  const long long n = (long long)count * c->nd;
  DevBuf qd, ud, ta, tb;
  CK(qd.ensure(sizeof(double) * n));
  CK(ud.ensure(sizeof(double) * n));
  CKS(copy_in(c, qd.p, q, sizeof(double) * n, where));
  if (c->opt.precision == RPA_FP64) {
    CK(ta.ensure(sizeof(double) * n));
    CK(tb.ensure(sizeof(double) * n));
    CKS((nu_half<double, double, double>(c, qd.as<double>(), c->nd, ud.as<double>(), count,
                                         ta.as<double>(), tb.as<double>())));
  } else {
    CK(ta.ensure(sizeof(float) * n));
    CK(tb.ensure(sizeof(float) * n));
    CKS((nu_half<float, double, double>(c, qd.as<double>(), c->nd, ud.as<double>(), count,
                                        ta.as<float>(), tb.as<float>())));
  }
  CKS(copy_out(c, u, ud.p, sizeof(double) * n, where));
  CK(cudaStreamSynchronize(c->stream));
  return RPA_OK;
}

rpa_status rpa_chi0(rpa_ctx* c, int count, const double* omega, const double* u, double* r,
                    int* iters, int where) {
  CKS(check_ready(c, false));
  if (count < 0 || (count > 0 && (!omega || !u || !r))) return fail(c, RPA_EINVAL, "bad arguments");
  if (count == 0) return RPA_OK;
  const int nb_max = choose_batch(c, count);
  CKS(ensure_workspace(c, nb_max));
  std::vector<double> om(count);
  if (where == RPA_DEVICE) {
    CK(cudaMemcpyAsync(om.data(), omega, sizeof(double) * count, cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
  } else
    std::memcpy(om.data(), omega, sizeof(double) * count);
  for (int i = 0; i < count; ++i)
    if (!(om[i] > 0.0)) return fail(c, RPA_EINVAL, "omega must be positive");
  c->soft = RPA_OK;
  for (int s0 = 0; s0 < count; s0 += nb_max) {
    const int nb = std::min(nb_max, count - s0);
    std::vector<int> ones(nb, 1);
    CK(cudaMemcpyAsync(c->active_d.p, ones.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->pomega_d.p, om.data() + s0, sizeof(double) * nb, cudaMemcpyHostToDevice,
                       c->stream));
    CKS(copy_in(c, c->u64.p, u + (long long)s0 * c->nd, sizeof(double) * nb * c->nd, where));
    SolveStats ss;
    if (c->opt.precision != RPA_FP64) {
      CK(convert_d2f(c->u64.as<double>(), c->u32.as<float>(), (long long)nb * c->nd, c->stream));
      CKS(solve_mixed(c, nb, c->u32.as<float>(), c->active_d.as<int>(), ss));
    } else {
      CKS(solve_fp64(c, nb, c->u64.as<double>(), c->active_d.as<int>(), ss));
    }
    if (ss.nonconv) note_soft(c, RPA_ENOCONV, "a Sternheimer solve reached stern_maxit");
    if (ss.breakdown)
      note_soft(c, RPA_EBREAKDOWN,
                "a COCG solve broke down (p^T A p = 0 or a non-finite residual)");
    CKS(copy_out(c, r + (long long)s0 * c->nd, c->dens64.p, sizeof(double) * nb * c->nd, where));
    if (iters) {
      std::vector<int> si((size_t)nb * c->ns * kSysI);
      CK(cudaMemcpyAsync(si.data(), c->sysi.p, sizeof(int) * si.size(), cudaMemcpyDeviceToHost,
                         c->stream));
      CK(cudaStreamSynchronize(c->stream));
      std::vector<int> it((size_t)nb * c->ns);
      for (size_t s = 0; s < it.size(); ++s) it[s] = si[s * kSysI + kIters];
      CKS(copy_out(c, iters + (long long)s0 * c->ns, it.data(), sizeof(int) * it.size(), where));
    }
    CK(cudaStreamSynchronize(c->stream));
  }
  return soft_status(c);
}

rpa_status rpa_galerkin(rpa_ctx* c, int count, const double* omega, const double* u, double* x0,
                        int where) {
  CKS(check_ready(c, false));
  if (count < 0 || (count > 0 && (!omega || !u || !x0))) return fail(c, RPA_EINVAL, "bad arguments");
  if (count == 0) return RPA_OK;
  const int nb_max = choose_batch(c, count);
  CKS(ensure_workspace(c, nb_max));
  std::vector<double> om(count);
  if (where == RPA_DEVICE) {
    CK(cudaMemcpyAsync(om.data(), omega, sizeof(double) * count, cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
  } else {
    std::memcpy(om.data(), omega, sizeof(double) * count);
  }
  const long long nd = c->nd;
  DevBuf xo;
  CK(xo.ensure(sizeof(cpx<double>) * (size_t)nb_max * c->ns * nd));
  CK(cudaMemsetAsync(c->flags_d.p, 0, sizeof(int) * 4, c->stream));
  for (int s0 = 0; s0 < count; s0 += nb_max) {
    const int nb = std::min(nb_max, count - s0);
    std::vector<int> ones(nb, 1);
    CK(cudaMemcpyAsync(c->active_d.p, ones.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->pomega_d.p, om.data() + s0, sizeof(double) * nb, cudaMemcpyHostToDevice,
                       c->stream));
    CKS(copy_in(c, c->u64.p, u + (long long)s0 * nd, sizeof(double) * nb * nd, where));
    const long long n = (long long)nb * c->ns * nd;
    if (c->opt.precision != RPA_FP64) {
      CK(convert_d2f(c->u64.as<double>(), c->u32.as<float>(), (long long)nb * nd, c->stream));
      CK(galerkin_guess_tc(nd, c->ns, nb, c->d32.psi.as<float>(), c->eps_d.as<double>(),
                           c->pomega_d.as<double>(), c->u32.as<float>(), c->active_d.as<int>(),
                           c->dV, c->gpart.as<double>(), gram_chunks(nd),
                           c->cmat.as<cpx<float>>(), c->x.as<cpx<float>>(),
                           c->flags_d.as<int>() + 2, c->stream,
                           c->opt.precision == RPA_MIXED_BF16, c->opt.debug_expire_waits));
      CK(convert_f2d(c->x.as<float>(), xo.as<double>(), 2 * n, c->stream));
    } else {
      CK(galerkin_guess<double>(nd, c->ns, nb, c->d64.psi.as<double>(), c->eps_d.as<double>(),
                                c->pomega_d.as<double>(), c->u64.as<double>(),
                                c->active_d.as<int>(), c->dV, c->gpart.as<double>(),
                                gram_chunks(nd), c->cmat.as<cpx<double>>(),
                                xo.as<cpx<double>>(), c->stream));
    }
    CKS(copy_out(c, x0 + 2 * (long long)s0 * c->ns * nd, xo.p, sizeof(cpx<double>) * n, where));
    CK(cudaStreamSynchronize(c->stream));
  }
  int flags[4];
  CK(cudaMemcpy(flags, c->flags_d.p, sizeof(flags), cudaMemcpyDeviceToHost));
  if (flags[2]) return fail(c, RPA_ETIMEOUT, "a bounded tensor-core wait expired");
  return RPA_OK;
}

rpa_status rpa_tridiag_f11(int count, int k, const double* alpha, const double* beta, int fkind,
                           double* d) {
  if (count < 0 || k < 1 || k > kMaxLanczos || (count > 0 && (!alpha || !beta || !d)) ||
      fkind < RPA_F_LOG || fkind > RPA_F_X2)
    return RPA_EINVAL;
  if (count == 0) return RPA_OK;
  double* buf = nullptr;
  const size_t n = (size_t)count * k;
  if (cudaMalloc(&buf, sizeof(double) * (2 * n + count)) != cudaSuccess) return RPA_ENOMEM;
  rpa_status st = RPA_OK;
  if (cudaMemcpy(buf, alpha, sizeof(double) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(buf + n, beta, sizeof(double) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
      tridiag_f11(count, k, buf, k, buf + n, k, nullptr, fkind, buf + 2 * n, 0) != cudaSuccess ||
      cudaMemcpy(d, buf + 2 * n, sizeof(double) * count, cudaMemcpyDeviceToHost) != cudaSuccess)
    st = RPA_ECUDA;
  cudaFree(buf);
  return st;
}

const char* rpa_status_string(rpa_status st) {
  switch (st) {
    case RPA_OK: return "ok";
    case RPA_EINVAL: return "invalid argument";
    case RPA_ENOMEM: return "out of memory";
    case RPA_ECUDA: return "CUDA error";
    case RPA_ENOCONV: return "Sternheimer solve did not converge";
    case RPA_EBREAKDOWN: return "breakdown";
    case RPA_ETIMEOUT: return "timeout";
    case RPA_ENOGAP: return "occupied set not separated";
    case RPA_ESTATE: return "call order";
  }
  return "unknown status";
}

const char* rpa_last_error(const rpa_ctx* c) { return c ? c->err.c_str() : "null context"; }

long long rpa_kernel_launches(const rpa_ctx*) { return g_launches.load(); }

}  // extern "C"
