/*
 * rpa.h -- C ABI of the GB300 library for the real-space RPA correlation energy by Lanczos
 * quadrature and interpolation.
 *
 * Method (paper: "Highly Parallel Real-Space Random Phase Approximation Using Lanczos
 * Quadrature and Interpolation"):
 *   E_c = 1/(2 pi) int_0^inf Tr[ log(I - nu chi0(i w)) + nu chi0(i w) ] dw          (Eq. 1)
 *       ~ 1/(2 pi) sum_k w_k sum_j d^_j(i w_k),  d^ = I_g(d on C_g)      (Eq. 9, Section 3.2)
 *   d_j(i w) = e_j^T f(A) e_j,  f(x) = log(1 - x) + x,  A = nu^{1/2} chi0(i w) nu^{1/2},
 *   approximated by [f(T_m)]_{11} after m Lanczos steps from e_j     (Eqs. 5-8, Algorithm 1)
 *   chi0(i w) u = 4 sum_n psi_n (.) Re(dpsi_n),
 *   (H - eps_n - i w) dpsi_n = -psi_n (.) u  solved by COCG with a Galerkin initial guess
 *                                                               (Eq. 4, Section 4)
 *   nu = -4 pi Lap_h^+ applied through the eigenbases of the 1-D finite-difference
 *   Laplacians (Kronecker-product formalism, Section 4).
 *
 * Conventions for every entry point:
 *   - Units are atomic (Hartree, bohr).  E_c is for the whole cell.
 *   - Grid vectors are flat arrays of N_d = nx*ny*nz values, x fastest:
 *     index = ix + nx*(iy + ny*iz).
 *   - Complex vectors are interleaved (re, im) pairs of doubles.
 *   - `where` (RPA_HOST or RPA_DEVICE) says where ALL pointer arguments of that call live.
 *     Device pointers must be device memory of the context's GPU and, for double data,
 *     8-byte aligned.
 *   - Ownership: the caller owns every buffer it passes; setters copy the data into
 *     library-owned device memory and keep no pointer to the caller's buffers.
 *   - All work is ordered on the context's CUDA stream; calls return after the results are
 *     in the caller's buffers (the call synchronises its stream).
 *   - Errors: every call returns an rpa_status; on failure rpa_last_error() gives a
 *     one-line reason.  The library never aborts or exits the process.  A CUDA error leaves
 *     the context unusable (RPA_ECUDA); destroy it.
 *   - Not thread-safe per context; distinct contexts may be used from distinct threads.
 */
#ifndef RPA_H_
#define RPA_H_

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RPA_OK = 0,
  RPA_EINVAL = 1,      /* bad argument or size */
  RPA_ENOMEM = 2,      /* device or host allocation failed */
  RPA_ECUDA = 3,       /* CUDA runtime error; context unusable */
  RPA_ENOCONV = 4,     /* a Sternheimer solve reached stern_maxit without convergence */
  RPA_EBREAKDOWN = 5,  /* COCG breakdown (p^T A p == 0) or non-finite Lanczos scalar */
  RPA_ETIMEOUT = 6,    /* a bounded device wait gave up */
  RPA_ENOGAP = 7,      /* occupied set not separated from the rest (eps not ascending) */
  RPA_ESTATE = 8       /* call order: a required setter has not been called */
} rpa_status;

enum { RPA_HOST = 0, RPA_DEVICE = 1 };
enum { RPA_PERIODIC = 0, RPA_DIRICHLET = 1 };
/* precision forms: plain FP64 everywhere, or FP32 stencil/COCG/projections with FP64
 * Lanczos basis, reorthogonalisation, tridiagonal eigen-solve, refinement residuals and
 * energy accumulation */
/* RPA_FP64: every step in FP64.  RPA_MIXED: FP32 stencil/COCG with FP64 residual refinement,
 * occupied-space projection GEMMs on the tensor cores in TF32x3 (fp32-level accuracy).
 * RPA_MIXED_BF16: as RPA_MIXED with single-pass BF16 projection GEMMs (FP32 accumulation). */
enum { RPA_FP64 = 0, RPA_MIXED = 1, RPA_MIXED_BF16 = 2 };
enum { RPA_INTERP_NONE = 0, RPA_INTERP_TRILINEAR = 1, RPA_INTERP_TRICUBIC = 2,
       RPA_INTERP_FOURIER = 3 };
/* matrix function hook (quadrature checks): f(x) = log(1-x)+x, x, or x^2 */
enum { RPA_F_LOG = 0, RPA_F_X = 1, RPA_F_X2 = 2 };

typedef struct rpa_ctx rpa_ctx;

/* Uniform finite-difference grid (Section 2, D1).  Spacings h[] in bohr; bc[a] periodic or
 * zero-Dirichlet per axis; fd_radius R gives the central Laplacian of order 2R (6 -> 12th
 * order).  Limits: 1 <= n[a] <= 1024, 1 <= fd_radius <= 8, nx*ny*nz < 2^31. */
typedef struct {
  int n[3];
  double h[3];
  int bc[3];
  int fd_radius;
} rpa_grid;

typedef struct {
  int lanczos_max;       /* N_l: matrix-vector products per probe (1..256) */
  double lanczos_rtol;   /* early exit when |d_k - d_{k-1}| <= rtol |d_k|, k >= 2; 0 = off */
  double stern_tol;      /* Sternheimer relative residual ||b - A x||_2 <= tol ||b||_2 */
  int stern_maxit;       /* COCG iteration cap per solve, counted over all refinement rounds
                            (RPA_ENOCONV beyond).  Default 20000: the solves at the smallest
                            frequencies grow with the cell and the tolerance (the iteration
                            tables of Section 5.6 rise as omega -> 0); a 64-atom cell at tol
                            1e-4 has needed several thousand, beyond an earlier default of
                            2000 */
  int precision;         /* RPA_FP64, RPA_MIXED or RPA_MIXED_BF16 */
  int reorth;            /* 1: full reorthogonalisation of the Lanczos basis (2 passes) */
  int stride[3];         /* coarsening factor g per axis (C_g of Section 3.2) */
  int interp;            /* RPA_INTERP_* */
  int batch;             /* probe-points in flight per wave; 0 = sized from free memory */
  int fkind;             /* RPA_F_* (RPA_F_LOG for the correlation energy) */
  int refine;            /* mixed form: FP64 residual refinement rounds after FP32 COCG */
  double inner_tol;      /* mixed form: FP32 COCG relative tolerance per round
                            (0 = auto: max(sqrt(stern_tol), 1e-5)) */
  int profile;           /* 1: time the COCG kernels with CUDA events (rpa_stats.kernel_*) */
  int tile;              /* xy tiling of the fused H-apply kernel: -1 = autotune (time the
                            candidate tilings on the first COCG solve of each precision and
                            keep the fastest), 0 = 32 x 8 column tiles, -2 = 64 x 8 tiles with
                            two x points per thread (mixed form, even nx), -3 / -4 = the same
                            with each thread's z window in a shared-memory ring instead of
                            registers (one / two centre-plane buffers), -6 = the two-point
                            kernel on packed full rows (mixed form, stencil radius 6, even nx
                            from 26 to 64; not among the autotuned candidates: on the 52^3
                            grid it measured within 1% of -2), h > 0 = tiles of h
                            full x rows (needs nx <= 64), -100 - h = bands of h full x rows with
                            two points per thread and a multi-stage asynchronous copy pipeline
                            (mixed form, even nx <= 64, h divides ny); RPA_EINVAL if it does not
                            fit */
  int graphs;            /* 2 (default): each COCG loop runs as one captured CUDA graph whose
                            conditional while nodes repeat chunks of fused iterations until
                            no system is active, the active list and counts rebuilt on the
                            device after every chunk (no host check inside the loop); with
                            profile = 1 one loop in four runs as with 1.  1: each chunk of
                            fused iterations is a captured graph replayed by the host, which
                            reads the active count after every chunk.  0: the kernels are
                            launched one by one */
  int lanczos_block;     /* 1: scalar Lanczos quadrature per probe (Section 3.1, default);
                            b in 2..8: block Lanczos quadrature, up to b consecutive probe-points
                            of one frequency and distinct grid points share one block
                            recurrence (the block variant named as future work in Section 6);
                            needs reorth = 1 and lanczos_rtol = 0; no tridiagonal output */
  int refine_restart;    /* mixed form, after each FP64 residual refinement: 0 = continue the
                            FP32 COCG recurrence from its last direction with the true
                            residual in place of the recursive one (a reliable update; the
                            Krylov space built so far is kept; default) when the inner
                            tolerance is >= 1e-3, else restart; 1 = always restart it from
                            p = r */
  int debug_expire_waits; /* tests only (default 0): 1 makes the first bounded wait of every
                            block of the tensor-core projection kernels (mixed form) wait on a
                            barrier that nothing arrives on, with a short limit, before any
                            MMA is issued; the call then returns RPA_ETIMEOUT with the tensor
                            memory freed and the context usable, so the bounded-wait failure
                            path can be tested without a GPU fault */
  int lanes;             /* 1 (default): the probe-points of a call run in waves one after
                            the other.  k in 2..8 (scalar Lanczos only): they are dealt
                            round-robin to k lanes that run concurrently, each with its own
                            CUDA stream, workspace and host thread (k - 1 helper contexts
                            created from this context's inputs on first use, dropped when an
                            input or option changes), so that the latency-bound COCG tail of
                            one lane overlaps the others' work; waves are sized from 1/k of
                            the free memory each.  Results and statistics are as for k = 1 */
} rpa_options;

typedef struct {
  double seconds_total;
  double seconds_phase[8]; /* 0 nu^{1/2}, 1 RHS + Galerkin projection, 2 COCG, 3 density,
                              4 Lanczos update, 5 tridiagonal f, 6 interpolation, 7 other */
  long long probe_points;  /* (probe, frequency) Lanczos runs completed */
  long long matvecs;       /* applications of A */
  long long solves;        /* Sternheimer systems solved */
  long long cocg_iters;    /* sum of COCG iterations over all solves */
  long long refine_rounds; /* FP64 refinement rounds (mixed form) */
  int max_cocg_iters;      /* largest iteration count of one solve */
  int lanczos_steps_max;   /* largest Lanczos step count of one probe */
  /* with options.profile: per COCG kernel class (0 projector dots, 1 H apply (matvec),
   * 2 scalar steps, 3 x/r update, 4 direction update) the summed event time, the number
   * of launches, and the algorithmic bytes moved (active systems x grid points x bytes per
   * point; projector data and scalars not counted).  Slots 5 and 6 of kernel_seconds: the
   * time of the sampled chunks whose launches covered at most 32 systems (the tail) and
   * more (the bulk); slots 5 and 6 of kernel_launches: those chunks' iterations */
  double kernel_seconds[8];
  long long kernel_launches[8];
  double kernel_bytes[8];
  int precision_bytes;     /* bytes of one real value in the COCG vectors (4 or 8) */
  int tile_rows;           /* tiling the H-apply kernel used for launches over many systems:
                              0 = 32 x 8 column tiles, -2 = 64 x 8 two-point tiles, h > 0 =
                              full-row tiles of height h */
  int tile_rows_tail;      /* the same for launches over at most 32 systems */
  long long nonconv_solves;   /* solves that ended above the tolerance (iteration cap, or
                                 refinement rounds or restarts used up) */
  long long breakdown_solves; /* solves that broke down (p^T A p = 0 or non-finite) */
} rpa_stats;

/* ---- context --------------------------------------------------------------------------- */

/* Create a context on the current CUDA device.  cuda_stream: a cudaStream_t to order all work
 * on, or NULL for a stream the library creates.  Computes the 1-D Laplacian eigenbases used
 * by nu^{1/2} on the device.  Errors: RPA_EINVAL (grid out of limits), RPA_ENOMEM, RPA_ECUDA. */
rpa_status rpa_create(rpa_ctx **out, const rpa_grid *grid, void *cuda_stream);
void rpa_destroy(rpa_ctx *ctx);

/* Local potential V_loc (N_d doubles, Ha). */
rpa_status rpa_set_potential(rpa_ctx *ctx, const double *vloc, int where);

/* Nonlocal projectors V_nl = sum_g sum_l gamma_{g,l} chi_{g,l} (dV chi_{g,l}^T .) grouped by
 * shared support (one group per atom for s/p projectors).  Host arrays only:
 *   nnz[g]: support size of group g; nproj[g]: projectors in group g (1..16);
 *   idx: concatenated supports (sum nnz ints, distinct grid indices within a group);
 *   chi: concatenated values, group-major then projector-major (sum nproj[g]*nnz[g]);
 *   gamma: concatenated coefficients (sum nproj[g], Ha).  ngroups = 0 clears V_nl. */
rpa_status rpa_set_projectors(rpa_ctx *ctx, int ngroups, const int *nnz, const int *nproj,
                              const int *idx, const double *chi, const double *gamma);

/* Occupied Kohn-Sham pairs (Eq. 3): psi is ns x N_d, state-major, normalised as
 * dV * sum_r psi_n(r)^2 = 1; eps ascending (RPA_ENOGAP otherwise).  1 <= ns <= 1024. */
rpa_status rpa_set_occupied(rpa_ctx *ctx, int ns, const double *psi, const double *eps,
                            int where);

/* Frequency nodes and weights of the outer quadrature (host arrays, 1 <= nw <= 64). */
rpa_status rpa_set_frequencies(rpa_ctx *ctx, int nw, const double *omega, const double *weight);

/* Gauss-Legendre rule of order nw mapped to [0, inf) by w = (1 + x)/(1 - x) with weights
 * 2 w_GL / (1 - x)^2 (Eq. 9), computed on the current device.  Host outputs. */
rpa_status rpa_gl_frequencies(int nw, double *omega, double *weight);

rpa_status rpa_default_options(rpa_options *opts);
rpa_status rpa_set_options(rpa_ctx *ctx, const rpa_options *opts);

/* Number of coarse probes P = |C_g| for the current stride, and their fine-grid indices
 * (x fastest over coarse nodes; host output of P long longs).  Coarse nodes per axis:
 * 0, g, 2g, ... plus n-1 on a Dirichlet axis. */
rpa_status rpa_num_probes(rpa_ctx *ctx, long long *nprobe);
rpa_status rpa_probe_indices(rpa_ctx *ctx, long long *idx);

/* ---- the hot path ---------------------------------------------------------------------- */

/* Algorithm 1 in full: d on C_g for every frequency, interpolation to the fine grid, E_c.
 * d_coarse (nw x P) and d_fine (nw x N_d) may be NULL.  ec: total E_c (Ha), may be NULL.
 * stats may be NULL.  Returns RPA_ENOCONV if any solve hit stern_maxit (results still
 * written). */
rpa_status rpa_energy_density(rpa_ctx *ctx, double *d_coarse, double *d_fine, double *ec,
                              rpa_stats *stats, int where);

/* Checkpoint file of rpa_energy_density (path copied; NULL or "" turns it off, the
 * default).  With a checkpoint, rpa_energy_density takes the (frequency, coarse point)
 * entries of d already in the file from it and computes only the others, in blocks of one
 * wave per lane; each block's entries are appended to the file (and flushed to the device)
 * as soon as the block completes, so a run that stops -- a killed job, a failed node --
 * loses at most the blocks in flight.  The file starts with a fingerprint of the problem
 * (grid, V_loc, projectors, occupied states and eigenvalues, frequencies, coarse set, and
 * the options that change d: lanczos_max, lanczos_rtol, stern_tol, stern_maxit, precision,
 * reorth, fkind, refine, inner_tol, lanczos_block, refine_restart); a file written for
 * another problem gives RPA_EINVAL and is left as it is.  A record cut short by a crash is
 * dropped on resume.  An entry's status (RPA_ENOCONV, RPA_EBREAKDOWN) is that of its block
 * and is reported again when the entry is resumed.  Contexts must not share a file.
 * Supports the paper's full-cell runs, which take hours (Section 5). */
rpa_status rpa_set_checkpoint(rpa_ctx *ctx, const char *path);

/* E_c of several independent systems (contexts of possibly different grids, boundary
 * conditions, occupied sets and options) in one call: each context runs rpa_energy_density
 * on its own stream from its own host thread, so their kernels overlap on the GPU.
 * ec_out (nsys doubles, host) receives each system's E_c; stats (nsys entries or NULL).
 * The contexts must be distinct.  Returns the first non-OK status of any system. */
rpa_status rpa_batch_energy(int nsys, rpa_ctx *const *sys, double *ec_out, rpa_stats *stats);

/* Lanczos quadrature for an explicit list of probe-points: probe[i] is a fine-grid index,
 * freq[i] an index into the frequency list.  d (count doubles) receives d_j(i w).  When
 * alpha/beta are non-NULL they receive the tridiagonal entries (count x lanczos_max, zero
 * padded; all zero with options.lanczos_block > 1, whose blocks are formed from consecutive
 * entries of one frequency) and steps (may be NULL) the step count per probe. */
rpa_status rpa_probe_density(rpa_ctx *ctx, int count, const long long *probe, const int *freq,
                             double *d, double *alpha, double *beta, int *steps,
                             rpa_stats *stats, int where);

/* Interpolation I_g of coarse values (nw x P) to the fine grid (nw x N_d, may be NULL) and
 * E_c = 1/(2 pi) sum_k w_k sum_j d^_j (ec may be NULL), with the context's options. */
rpa_status rpa_interpolate(rpa_ctx *ctx, const double *d_coarse, double *d_fine, double *ec,
                           int where);

/* ---- single steps of the path (each runs on the GPU; used by parity tests) -------------- */

/* y_i = (H - sigma_i) x_i for count complex vectors (count x N_d interleaved); sigma: count
 * complex shifts (interleaved).  Runs in the context's precision form. */
rpa_status rpa_apply_h(rpa_ctx *ctx, int count, const double *x, const double *sigma,
                       double *y, int where);

/* u_i = nu^{1/2} q_i for count real vectors (count x N_d). */
rpa_status rpa_apply_nu_half(rpa_ctx *ctx, int count, const double *q, double *u, int where);

/* r_i = chi0(i omega_i) u_i by the N_s Sternheimer solves (count x N_d real); iters (may be
 * NULL) receives count x N_s COCG iteration counts. */
rpa_status rpa_chi0(rpa_ctx *ctx, int count, const double *omega, const double *u, double *r,
                    int *iters, int where);

/* Galerkin initial guesses of the Sternheimer systems (Section 4): for each of count
 * (omega_i, u_i) and each occupied state n, x0_{i,n} = sum_k psi_k C_kn with
 * C_kn = dV psi_k^T(-psi_n (.) u_i) / (eps_k - eps_n - i omega_i).  u: count x N_d real;
 * x0: count x N_s x N_d complex (interleaved).  Mixed form: tcgen05 tensor cores (tf32,
 * three-pass split); FP64 form: FP64 CUDA cores. */
rpa_status rpa_galerkin(rpa_ctx *ctx, int count, const double *omega, const double *u,
                        double *x0, int where);

/* Galerkin initial guesses (as rpa_galerkin in the FP64 form) for callers that cannot
 * allocate device memory themselves -- for instance code running under another framework's
 * memory pool, or a path that must avoid cudaMalloc/cudaFree because they synchronise the
 * whole device.  The paper has no counterpart; this is a service of the library.
 *   All pointers are DEVICE pointers of the current device: psi (ns x nd, state-major,
 *   dV sum psi^2 = 1), eps (ns), omega (count), u (count x nd real), x0 (count x ns x nd
 *   complex, interleaved) -- the caller owns and allocates them.  dV: volume element.
 *   Work is queued on cuda_stream (NULL: the legacy default stream) and the call returns
 *   without synchronising; read x0 after synchronising that stream.
 *   Scratch: a fixed 8 MiB file-scope device array (held by every GPU that loads the library
 *   until exit); needs ceil(nd/4096) (clamped to 1..256) x ns^2 x 8 bytes (rounded up to a
 *   multiple of 256) + ns^2 x 16 bytes, e.g.
 *   35 x 128^2 x 8 + 128^2 x 16 = 4.85 MB for a 52^3 grid with 128 states.  Larger sizes are
 *   rejected with RPA_EINVAL before any work is queued.
 *   Every call made outside a stream capture looks up the array's device address
 *   (cudaGetSymbolAddress) on the current device; a call inside a capture reuses the address
 *   of the last uncaptured call on that device (RPA_ECUDA if there was none), so make one
 *   call before any stream capture.  The call allocates nothing (no
 *   cudaMalloc, no cudaFree).  Every call shares the scratch array and leaves its contents
 *   behind; calls whose work overlaps on the GPU (different streams, or host threads
 *   without ordering) race on it and must be serialised by the caller. */
rpa_status rpa_galerkin_noalloc(long long nd, int ns, const double *psi, const double *eps,
                                double dV, int count, const double *omega, const double *u,
                                double *x0, void *cuda_stream);

/* d_i = [f(T_i)]_{11} for count symmetric tridiagonals of order k (alpha: count x k,
 * beta: count x k with beta[i*k + k-1] ignored); host arrays; solved on the device. */
rpa_status rpa_tridiag_f11(int count, int k, const double *alpha, const double *beta,
                           int fkind, double *d);

const char *rpa_status_string(rpa_status st);
const char *rpa_last_error(const rpa_ctx *ctx);
/* Number of kernels this context has launched since creation (launch accounting). */
long long rpa_kernel_launches(const rpa_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* RPA_H_ */
