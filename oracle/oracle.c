/*
 * Oracle for the RPA correlation-energy density by Lanczos quadrature (CPU, FP64).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, literal CPU restatement of the
 * method of "Highly Parallel Real-Space Random Phase Approximation Using Lanczos Quadrature
 * and Interpolation" (Algorithm 1 and Eqs. 1-9).  It exists so that the CUDA library can be
 * checked against something independent.  Only the test-suite, the package smoke check and
 * the CPU baseline of the benchmark load it; the product path never does.  It shares no code,
 * header, table or constant generator with the CUDA library.
 *
 * Conventions (atomic units):
 *   grid n[0] x n[1] x n[2], flat index ix + nx*(iy + ny*iz), spacings h[], volume element
 *   dV = hx*hy*hz; bc[a] = 0 periodic, 1 zero-Dirichlet (zero ghost values).
 *   Lap_h = central finite-difference Laplacian of radius R (order 2R), Section 2.
 *   H = -1/2 Lap_h + diag(vloc) + sum_p gamma_p chi_p (dV chi_p^T .)   (Eq. 3's operator)
 *   Orbitals psi_n normalised as dV * sum psi_n^2 = 1.
 *   nu = -4 pi Lap_h^+ (pseudo-inverse on the range for periodic cells); nu^{1/2} is its PSD
 *   square root, applied in the eigenbasis of Lap_h = Lx (+) Ly (+) Lz (Kronecker sum),
 *   i.e. by three 1-D mode products each way (Section 4, Kronecker-product formalism).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

typedef struct {
  int n[3];
  double h[3];
  int bc[3];
  int radius;
  const double *vloc;       /* N_d */
  int nproj;                /* projectors */
  const int *proj_off;      /* nproj + 1 offsets into proj_idx / proj_val */
  const int *proj_idx;      /* grid indices of each projector's support */
  const double *proj_val;   /* projector values on its support */
  const double *proj_gamma; /* nproj coefficients (Ha) */
  int ns;                   /* occupied states N_s */
  const double *psi;        /* ns x N_d, state-major */
  const double *eps;        /* ns */
} orc_sys;

typedef struct {
  int nl;        /* Lanczos steps N_l (matrix-vector products per probe) */
  double lrtol;  /* early exit when |d_k - d_{k-1}| <= lrtol |d_k| (k >= 2); 0 disables */
  double tol;    /* Sternheimer relative residual ||b - A x||_2 <= tol ||b||_2 */
  int maxit;     /* COCG iteration cap per solve */
  int reorth;    /* 1: full reorthogonalisation of the Lanczos basis (two Gram-Schmidt passes) */
  int fkind;     /* 0: f(x) = log(1-x) + x;  1: f(x) = x;  2: f(x) = x^2 (quadrature checks) */
  int nthreads;  /* OpenMP threads, 0 = default */
} orc_opts;

static long nd_of(const orc_sys *s) { return (long)s->n[0] * s->n[1] * s->n[2]; }
static double dv_of(const orc_sys *s) { return s->h[0] * s->h[1] * s->h[2]; }

/* ---------------------------------------------------------------------------------------
 * Central second-derivative weights of radius R (order 2R), closed form:
 *   c_m = 2 (-1)^{m+1} (R!)^2 / (m^2 (R-m)! (R+m)!),  c_0 = -2 sum_{m>=1} c_m.
 * ------------------------------------------------------------------------------------- */
void orc_fd_weights(int R, double *c) {
  double fR = 1.0;
  for (int i = 2; i <= R; ++i) fR *= i;
  double s = 0.0;
  for (int m = 1; m <= R; ++m) {
    double fm = 1.0, fp = 1.0;
    for (int i = 2; i <= R - m; ++i) fm *= i;
    for (int i = 2; i <= R + m; ++i) fp *= i;
    double v = 2.0 * fR * fR / ((double)m * m * fm * fp);
    c[m] = (m % 2 == 1) ? v : -v;
    s += c[m];
  }
  c[0] = -2.0 * s;
}

/* neighbour index along one axis; -1 when it falls outside a Dirichlet axis */
static int shift_index(int i, int m, int n, int bc) {
  int j = i + m;
  if (bc == 0) {
    j %= n;
    if (j < 0) j += n;
    return j;
  }
  return (j < 0 || j >= n) ? -1 : j;
}

/* y = (H - sigma) x for complex x (Eq. 4's operator with sigma = eps_n + i omega). */
void orc_apply_h(const orc_sys *s, const cplx *x, cplx sigma, cplx *y) {
  const int nx = s->n[0], ny = s->n[1], nz = s->n[2];
  const long N = nd_of(s);
  double c[32];
  orc_fd_weights(s->radius, c);
  const double ax = -0.5 / (s->h[0] * s->h[0]);
  const double ay = -0.5 / (s->h[1] * s->h[1]);
  const double az = -0.5 / (s->h[2] * s->h[2]);
  for (int iz = 0; iz < nz; ++iz)
    for (int iy = 0; iy < ny; ++iy)
      for (int ix = 0; ix < nx; ++ix) {
        long p = ix + (long)nx * (iy + (long)ny * iz);
        cplx acc = (c[0] * (ax + ay + az) + s->vloc[p] - sigma) * x[p];
        for (int m = 1; m <= s->radius; ++m) {
          for (int sg = -1; sg <= 1; sg += 2) {
            int jx = shift_index(ix, sg * m, nx, s->bc[0]);
            int jy = shift_index(iy, sg * m, ny, s->bc[1]);
            int jz = shift_index(iz, sg * m, nz, s->bc[2]);
            if (jx >= 0) acc += ax * c[m] * x[jx + (long)nx * (iy + (long)ny * iz)];
            if (jy >= 0) acc += ay * c[m] * x[ix + (long)nx * (jy + (long)ny * iz)];
            if (jz >= 0) acc += az * c[m] * x[ix + (long)nx * (iy + (long)ny * jz)];
          }
        }
        y[p] = acc;
      }
  const double dV = dv_of(s);
  for (int q = 0; q < s->nproj; ++q) {
    cplx dot = 0.0;
    for (int e = s->proj_off[q]; e < s->proj_off[q + 1]; ++e) dot += s->proj_val[e] * x[s->proj_idx[e]];
    dot *= s->proj_gamma[q] * dV;
    for (int e = s->proj_off[q]; e < s->proj_off[q + 1]; ++e) y[s->proj_idx[e]] += s->proj_val[e] * dot;
  }
  (void)N;
}

/* ---------------------------------------------------------------------------------------
 * Symmetric eigen-decomposition by cyclic Jacobi rotations (dense, small n).
 * a: n x n row-major, destroyed; lam: n eigenvalues; v: n x n, column i = eigenvector i.
 * ------------------------------------------------------------------------------------- */
void orc_jacobi_eig(int n, double *a, double *lam, double *v) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) v[i * n + j] = (i == j) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        tot += a[i * n + j] * a[i * n + j];
        if (i != j) off += a[i * n + j] * a[i * n + j];
      }
    if (off <= 1e-30 * tot || off == 0.0) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = a[p * n + q];
        if (apq == 0.0) continue;
        double app = a[p * n + p], aqq = a[q * n + q];
        /* rotation angle that zeroes a_pq: tan(2 theta) = 2 a_pq / (a_qq - a_pp) */
        double theta = 0.5 * atan2(2.0 * apq, aqq - app);
        double cs = cos(theta), sn = sin(theta);
        for (int k = 0; k < n; ++k) { /* columns p, q */
          double akp = a[k * n + p], akq = a[k * n + q];
          a[k * n + p] = cs * akp - sn * akq;
          a[k * n + q] = sn * akp + cs * akq;
        }
        for (int k = 0; k < n; ++k) { /* rows p, q */
          double apk = a[p * n + k], aqk = a[q * n + k];
          a[p * n + k] = cs * apk - sn * aqk;
          a[q * n + k] = sn * apk + cs * aqk;
        }
        for (int k = 0; k < n; ++k) {
          double vkp = v[k * n + p], vkq = v[k * n + q];
          v[k * n + p] = cs * vkp - sn * vkq;
          v[k * n + q] = sn * vkp + cs * vkq;
        }
      }
  }
  for (int i = 0; i < n; ++i) lam[i] = a[i * n + i];
}

/* 1-D finite-difference second-derivative matrix (1/h^2 scaled) and its eigenpairs. */
void orc_lap1d_eig(int n, double h, int bc, int R, double *V, double *lam) {
  double c[32];
  orc_fd_weights(R, c);
  double *a = (double *)calloc((size_t)n * n, sizeof(double));
  for (int i = 0; i < n; ++i) {
    a[i * n + i] += c[0] / (h * h);
    for (int m = 1; m <= R; ++m)
      for (int sg = -1; sg <= 1; sg += 2) {
        int j = shift_index(i, sg * m, n, bc);
        if (j >= 0) a[i * n + j] += c[m] / (h * h);
      }
  }
  orc_jacobi_eig(n, a, lam, V);
  free(a);
}

typedef struct {
  int n[3];
  double *V[3];   /* eigenvectors, n x n, column k = mode k */
  double *lam[3];
  double *scale;  /* N_d: sqrt(4 pi / -(lx + ly + lz)), 0 on the null space */
} orc_nu;

static void nu_init(const orc_sys *s, orc_nu *nu) {
  double lmax = 0.0;
  for (int a = 0; a < 3; ++a) {
    int n = s->n[a];
    nu->n[a] = n;
    nu->V[a] = (double *)malloc(sizeof(double) * n * n);
    nu->lam[a] = (double *)malloc(sizeof(double) * n);
    orc_lap1d_eig(n, s->h[a], s->bc[a], s->radius, nu->V[a], nu->lam[a]);
    double m = 0.0;
    for (int i = 0; i < n; ++i) m = fmax(m, fabs(nu->lam[a][i]));
    lmax += m;
  }
  long N = nd_of(s);
  nu->scale = (double *)malloc(sizeof(double) * N);
  for (int k = 0; k < s->n[2]; ++k)
    for (int j = 0; j < s->n[1]; ++j)
      for (int i = 0; i < s->n[0]; ++i) {
        double neg = -(nu->lam[0][i] + nu->lam[1][j] + nu->lam[2][k]);
        long p = i + (long)s->n[0] * (j + (long)s->n[1] * k);
        nu->scale[p] = (neg > 1e-10 * lmax) ? sqrt(4.0 * M_PI / neg) : 0.0;
      }
}

static void nu_free(orc_nu *nu) {
  for (int a = 0; a < 3; ++a) { free(nu->V[a]); free(nu->lam[a]); }
  free(nu->scale);
}

/* out = (Vz (x) Vy (x) Vx)^{T or not} in, along each axis (mode products). */
static void mode_products(const orc_nu *nu, const double *in, double *out, int transpose) {
  const int nx = nu->n[0], ny = nu->n[1], nz = nu->n[2];
  const long N = (long)nx * ny * nz;
  double *t1 = (double *)malloc(sizeof(double) * N), *t2 = (double *)malloc(sizeof(double) * N);
  /* x axis */
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int a = 0; a < nx; ++a) {
        double acc = 0.0;
        for (int i = 0; i < nx; ++i) {
          double m = transpose ? nu->V[0][i * nx + a] : nu->V[0][a * nx + i];
          acc += m * in[i + (long)nx * (j + (long)ny * k)];
        }
        t1[a + (long)nx * (j + (long)ny * k)] = acc;
      }
  /* y axis */
  for (int k = 0; k < nz; ++k)
    for (int b = 0; b < ny; ++b)
      for (int i = 0; i < nx; ++i) {
        double acc = 0.0;
        for (int j = 0; j < ny; ++j) {
          double m = transpose ? nu->V[1][j * ny + b] : nu->V[1][b * ny + j];
          acc += m * t1[i + (long)nx * (j + (long)ny * k)];
        }
        t2[i + (long)nx * (b + (long)ny * k)] = acc;
      }
  /* z axis */
  for (int c = 0; c < nz; ++c)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        double acc = 0.0;
        for (int k = 0; k < nz; ++k) {
          double m = transpose ? nu->V[2][k * nz + c] : nu->V[2][c * nz + k];
          acc += m * t2[i + (long)nx * (j + (long)ny * k)];
        }
        out[i + (long)nx * (j + (long)ny * c)] = acc;
      }
  free(t1);
  free(t2);
}

/* u = nu^{1/2} q (Section 4; symmetric PSD square root of -4 pi Lap_h^+). */
static void nu_half_apply(const orc_nu *nu, const double *q, double *u) {
  const long N = (long)nu->n[0] * nu->n[1] * nu->n[2];
  double *t = (double *)malloc(sizeof(double) * N);
  mode_products(nu, q, t, 1);
  for (long p = 0; p < N; ++p) t[p] *= nu->scale[p];
  mode_products(nu, t, u, 0);
  free(t);
}

void orc_nu_half(const orc_sys *s, int count, const double *q, double *u) {
  orc_nu nu;
  nu_init(s, &nu);
  const long N = nd_of(s);
  for (int i = 0; i < count; ++i) nu_half_apply(&nu, q + i * N, u + i * N);
  nu_free(&nu);
}

/* ---------------------------------------------------------------------------------------
 * Sternheimer solve (Eq. 4) by COCG with a Galerkin initial guess (Section 4):
 *   (H - eps_n - i omega) x = b,  b = -psi_n (.) u.
 * Galerkin guess: the exact solution restricted to span{psi_k}:
 *   x0 = sum_k psi_k C_k,  C_k = dV psi_k^T b / (eps_k - eps_n - i omega).
 * COCG uses the unconjugated bilinear form a^T b; it stops when the recursive residual
 * satisfies ||r||_2 <= tol ||b||_2 and then re-checks the true residual, restarting from the
 * current iterate if the true residual is still above tol.  Returns iterations taken, or
 * -1 when maxit is exhausted, or -2 when 50 restarts end with the true residual still
 * above tol (the stopping rule of Section 4 was not met).
 * ------------------------------------------------------------------------------------- */
static double norm2c(const cplx *a, long N) {
  double s = 0.0;
  for (long i = 0; i < N; ++i) s += creal(a[i]) * creal(a[i]) + cimag(a[i]) * cimag(a[i]);
  return sqrt(s);
}

static cplx dotu(const cplx *a, const cplx *b, long N) {
  cplx s = 0.0;
  for (long i = 0; i < N; ++i) s += a[i] * b[i];
  return s;
}

static int cocg_solve(const orc_sys *s, int n, double omega, const double *u, double tol,
                      int maxit, cplx *x, cplx *b, cplx *r, cplx *p, cplx *w) {
  const long N = nd_of(s);
  const double dV = dv_of(s);
  const cplx sigma = s->eps[n] + I * omega;
  const double *psin = s->psi + (long)n * N;
  for (long i = 0; i < N; ++i) b[i] = -psin[i] * u[i];
  /* Galerkin initial guess over the occupied space */
  for (long i = 0; i < N; ++i) x[i] = 0.0;
  for (int k = 0; k < s->ns; ++k) {
    const double *psik = s->psi + (long)k * N;
    cplx g = 0.0;
    for (long i = 0; i < N; ++i) g += psik[i] * b[i];
    g *= dV;
    cplx ck = g / (s->eps[k] - sigma);
    for (long i = 0; i < N; ++i) x[i] += ck * psik[i];
  }
  const double bn = norm2c(b, N);
  if (bn == 0.0) return 0;
  int it = 0;
  for (int restart = 0; restart < 50; ++restart) {
    orc_apply_h(s, x, sigma, w);
    for (long i = 0; i < N; ++i) { r[i] = b[i] - w[i]; p[i] = r[i]; }
    if (norm2c(r, N) <= tol * bn) return it;
    cplx rho = dotu(r, r, N);
    for (;;) {
      if (it >= maxit) return -1;
      orc_apply_h(s, p, sigma, w);
      cplx mu = dotu(p, w, N);
      if (mu == 0.0) return -1;
      cplx alpha = rho / mu;
      for (long i = 0; i < N; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * w[i]; }
      ++it;
      if (norm2c(r, N) <= tol * bn) break;
      cplx rho1 = dotu(r, r, N);
      cplx beta = rho1 / rho;
      rho = rho1;
      for (long i = 0; i < N; ++i) p[i] = r[i] + beta * p[i];
    }
  }
  /* every restart converged recursively but the true residual never met the tolerance */
  orc_apply_h(s, x, sigma, w);
  for (long i = 0; i < N; ++i) r[i] = b[i] - w[i];
  return norm2c(r, N) <= tol * bn ? it : -2;
}

/* Galerkin initial guesses of all N_s systems for one u (Section 4):
 * x0_n = sum_k psi_k C_kn,  C_kn = dV psi_k^T (-psi_n u) / (eps_k - eps_n - i omega).
 * x0: ns x N_d complex (interleaved).  Exported for tests of the projection step. */
void orc_galerkin(const orc_sys *s, double omega, const double *u, double *x0out) {
  const long N = nd_of(s);
  const double dV = dv_of(s);
  cplx *x0 = (cplx *)x0out;
  for (int n = 0; n < s->ns; ++n) {
    const double *psin = s->psi + (long)n * N;
    cplx *xn = x0 + (long)n * N;
    for (long i = 0; i < N; ++i) xn[i] = 0.0;
    for (int k = 0; k < s->ns; ++k) {
      const double *psik = s->psi + (long)k * N;
      double g = 0.0;
      for (long i = 0; i < N; ++i) g += psik[i] * (-psin[i] * u[i]);
      cplx ck = g * dV / (s->eps[k] - s->eps[n] - I * omega);
      for (long i = 0; i < N; ++i) xn[i] += ck * psik[i];
    }
  }
}

/* r = chi0(i omega) u via the N_s Sternheimer solves: r = 4 sum_n psi_n (.) Re(dpsi_n)
 * (Algorithm 1, inner loop over occupied states).  Solves run in parallel; the density is
 * summed over n in order afterwards.  iters[n] receives each solve's COCG iterations. */
static int chi0_apply(const orc_sys *s, double omega, const double *u, double tol, int maxit,
                      double *r, int *iters, double *xre_all) {
  const long N = nd_of(s);
  int fail = 0;
#pragma omp parallel
  {
    cplx *x = (cplx *)malloc(sizeof(cplx) * N * 5);
    cplx *b = x + N, *rr = x + 2 * N, *p = x + 3 * N, *w = x + 4 * N;
#pragma omp for schedule(dynamic, 1)
    for (int n = 0; n < s->ns; ++n) {
      int it = cocg_solve(s, n, omega, u, tol, maxit, x, b, rr, p, w);
      if (it < 0) {
#pragma omp atomic write
        fail = 1;
      }
      iters[n] = it;
      for (long i = 0; i < N; ++i) xre_all[(long)n * N + i] = creal(x[i]);
    }
    free(x);
  }
  for (long i = 0; i < N; ++i) r[i] = 0.0;
  for (int n = 0; n < s->ns; ++n) {
    const double *psin = s->psi + (long)n * N;
    for (long i = 0; i < N; ++i) r[i] += 4.0 * psin[i] * xre_all[(long)n * N + i];
  }
  return fail ? -1 : 0;
}

/* public: r = chi0(i omega) u for one vector u (tests of the Sternheimer step). */
int orc_chi0(const orc_sys *s, double omega, const double *u, double tol, int maxit, int nthreads,
             double *r, int *iters) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
  const long N = nd_of(s);
  double *xre = (double *)malloc(sizeof(double) * N * s->ns);
  int st = chi0_apply(s, omega, u, tol, maxit, r, iters, xre);
  free(xre);
  return st;
}

/* ---------------------------------------------------------------------------------------
 * [f(T)]_{11} of the symmetric tridiagonal T (diagonal al[0..k-1], off-diagonal be[0..k-2])
 * = sum_i Q_{1i}^2 f(lambda_i) with T Q = Q Lambda (Eq. 7, Algorithm 1).
 * ------------------------------------------------------------------------------------- */
static double fval(double x, int fkind) {
  if (fkind == 1) return x;
  if (fkind == 2) return x * x;
  return log1p(-x) + x;
}

double orc_tridiag_f11(int k, const double *al, const double *be, int fkind) {
  double *a = (double *)calloc((size_t)k * k, sizeof(double));
  double *v = (double *)malloc(sizeof(double) * k * k);
  double *lam = (double *)malloc(sizeof(double) * k);
  for (int i = 0; i < k; ++i) {
    a[i * k + i] = al[i];
    if (i + 1 < k) { a[i * k + i + 1] = be[i]; a[(i + 1) * k + i] = be[i]; }
  }
  orc_jacobi_eig(k, a, lam, v);
  double d = 0.0;
  for (int i = 0; i < k; ++i) d += v[i] * v[i] * fval(lam[i], fkind); /* v[0*k + i] = Q_{1i} */
  free(a); free(v); free(lam);
  return d;
}

/* ---------------------------------------------------------------------------------------
 * Lanczos quadrature of one diagonal entry d_j(i omega) = e_j^T f(A) e_j,
 * A = nu^{1/2} chi0(i omega) nu^{1/2} (Section 3.1, Algorithm 1):
 *   q_1 = e_j, beta_0 = 0; for k = 1..N_l: v = A q_k; alpha_k = q_k^T v;
 *   v -= alpha_k q_k + beta_{k-1} q_{k-1}; [full reorthogonalisation];
 *   if k < N_l: beta_k = ||v||, q_{k+1} = v / beta_k.
 * Then d = [f(T)]_{11}.  Early exit (optional) and breakdown (beta_k <= 1e-14 |alpha_1|)
 * stop with the tridiagonal built so far.
 * ------------------------------------------------------------------------------------- */
static int lanczos_probe(const orc_sys *s, const orc_nu *nu, const orc_opts *o, long j,
                         double omega, double *d_out, double *al, double *be, long *cocg_iters,
                         double *Q, double *v, double *u, double *r, double *xre, int *iters) {
  const long N = nd_of(s);
  for (long i = 0; i < N; ++i) Q[i] = 0.0;
  Q[j] = 1.0;
  double dprev = 0.0, d = 0.0;
  int steps = 0, status = 0;
  *cocg_iters = 0;
  for (int k = 0; k < o->nl; ++k) {
    const double *qk = Q + (long)k * N;
    /* v = nu^{1/2} chi0 nu^{1/2} q_k, matrix-free */
    nu_half_apply(nu, qk, u);
    if (chi0_apply(s, omega, u, o->tol, o->maxit, r, iters, xre) != 0) status = 1;
    for (int n = 0; n < s->ns; ++n) *cocg_iters += iters[n] > 0 ? iters[n] : 0;
    nu_half_apply(nu, r, v);
    double a = 0.0;
    for (long i = 0; i < N; ++i) a += qk[i] * v[i];
    al[k] = a;
    for (long i = 0; i < N; ++i) v[i] -= a * qk[i];
    if (k > 0) {
      const double *qp = Q + (long)(k - 1) * N;
      for (long i = 0; i < N; ++i) v[i] -= be[k - 1] * qp[i];
    }
    if (o->reorth) {
      for (int pass = 0; pass < 2; ++pass) {
        double cs[512];
        for (int m = 0; m <= k; ++m) {
          const double *qm = Q + (long)m * N;
          double c = 0.0;
          for (long i = 0; i < N; ++i) c += qm[i] * v[i];
          cs[m] = c;
        }
        for (int m = 0; m <= k; ++m) {
          const double *qm = Q + (long)m * N;
          for (long i = 0; i < N; ++i) v[i] -= cs[m] * qm[i];
        }
      }
    }
    steps = k + 1;
    if (o->lrtol > 0.0 || k == o->nl - 1) {
      d = orc_tridiag_f11(steps, al, be, o->fkind);
      if (o->lrtol > 0.0 && k >= 1 && fabs(d - dprev) <= o->lrtol * fabs(d)) break;
      dprev = d;
    }
    if (k < o->nl - 1) {
      double bn = 0.0;
      for (long i = 0; i < N; ++i) bn += v[i] * v[i];
      bn = sqrt(bn);
      if (bn <= 1e-14 * fabs(al[0]) || bn == 0.0) {
        d = orc_tridiag_f11(steps, al, be, o->fkind);
        break;
      }
      be[k] = bn;
      double *qn = Q + (long)(k + 1) * N;
      for (long i = 0; i < N; ++i) qn[i] = v[i] / bn;
    }
  }
  *d_out = d;
  return status ? -steps : steps;
}

/* Batch of probe-points: grid index probe[i] at frequency omega[i].  Outputs per probe:
 * d[i], steps[i] (negative when a Sternheimer solve hit maxit), alpha/beta (count x nl),
 * total COCG iterations. */
int orc_lanczos_batch(const orc_sys *s, const orc_opts *o, int count, const long *probe,
                      const double *omega, double *d, int *steps, double *alpha, double *beta,
                      long *cocg_iters) {
#ifdef _OPENMP
  if (o->nthreads > 0) omp_set_num_threads(o->nthreads);
#endif
  if (o->nl > 512) return -1;
  orc_nu nu;
  nu_init(s, &nu);
  const long N = nd_of(s);
  double *Q = (double *)malloc(sizeof(double) * N * (o->nl + 1));
  double *v = (double *)malloc(sizeof(double) * N * 3);
  double *u = v + N, *r = v + 2 * N;
  double *xre = (double *)malloc(sizeof(double) * N * s->ns);
  int *iters = (int *)malloc(sizeof(int) * s->ns);
  int bad = 0;
  for (int i = 0; i < count; ++i) {
    for (int k = 0; k < o->nl; ++k) { alpha[(long)i * o->nl + k] = 0.0; beta[(long)i * o->nl + k] = 0.0; }
    steps[i] = lanczos_probe(s, &nu, o, probe[i], omega[i], &d[i], alpha + (long)i * o->nl,
                             beta + (long)i * o->nl, &cocg_iters[i], Q, v, u, r, xre, iters);
    if (steps[i] < 0) bad = 1;
  }
  free(Q); free(v); free(xre); free(iters);
  nu_free(&nu);
  return bad ? 1 : 0;
}

/* y = (H - sigma) x for `count` complex vectors (interleaved re/im), for tests. */
void orc_apply_h_batch(const orc_sys *s, int count, const double *x, double sig_re,
                       double sig_im, double *y) {
  const long N = nd_of(s);
  for (int i = 0; i < count; ++i)
    orc_apply_h(s, (const cplx *)(x + 2 * N * i), sig_re + I * sig_im, (cplx *)(y + 2 * N * i));
}

/* 1-D eigenpairs used by nu^{1/2}, exported for tests. */
void orc_nu_modes(const orc_sys *s, int axis, double *V, double *lam) {
  orc_lap1d_eig(s->n[axis], s->h[axis], s->bc[axis], s->radius, V, lam);
}

/* ---------------------------------------------------------------------------------------
 * Gauss-Legendre nodes on [-1, 1] by Newton iteration on P_n (three-term recurrence), mapped
 * to [0, inf) by omega = (1 + x) / (1 - x), weight 2 w / (1 - x)^2 (Eq. 9; the mapping is the
 * one that reproduces the frequencies printed in the COCG-iteration tables).
 * ------------------------------------------------------------------------------------- */
void orc_gl_frequencies(int nw, double *omega, double *weight) {
  for (int i = 0; i < nw; ++i) {
    double x = cos(M_PI * (i + 0.75) / (nw + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= nw; ++k) {
        double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (nw == 1) { p1 = x; p0 = 1.0; }
      dp = nw * (x * p1 - p0) / (x * x - 1.0);
      double dx = p1 / dp;
      x -= dx;
      if (fabs(dx) < 1e-16) break;
    }
    {
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= nw; ++k) {
        double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (nw == 1) { p1 = x; p0 = 1.0; }
      dp = nw * (x * p1 - p0) / (x * x - 1.0);
    }
    double w = 2.0 / ((1.0 - x * x) * dp * dp);
    omega[i] = (1.0 + x) / (1.0 - x);
    weight[i] = 2.0 * w / ((1.0 - x) * (1.0 - x));
  }
}
