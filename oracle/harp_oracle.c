/*
 * harp_oracle.c -- plain FP64 CPU oracle for the HARP fill and the MBF solve.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, obviously correct
 * definition that the CUDA path is checked against. Only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark may load it. It
 * shares no code, header, table or helper with the CUDA library.
 *
 * What it computes (Bui-Van et al., "Fast and Accurate Simulation Technique
 * for Large Irregular Arrays", Section II):
 *
 *   Eq. 1  far-field term    Z_app = -j w mu0 g_TS(alpha) e^{-jkr} / (4 pi r)
 *   Eq. 3  HARP series       B_TS  = sum_{p=-P..P} e^{j p alpha} sum_{q=0..Q} c_pq^{TS} d^q
 *          with d = 1/r (the improved change of variables of Section II-B;
 *          d = 1/r^2 of the original model is kept as a variant)
 *   Eq. 4  interaction       Z_TS  = Z_app + B_TS e^{-jkr}
 *
 * for every ordered antenna pair m != n, with r = |x_m - x_n| and alpha the
 * direction from the source antenna n to the testing antenna m, measured
 * anticlockwise from +x. Diagonal blocks are the caller's self blocks,
 * copied. The reduced matrix is then solved for every port excitation by a
 * textbook LU factorisation with partial pivoting (the O((Na Nm)^3) direct
 * solve of Section II-B), forward and back substitution.
 *
 * Layouts: complex numbers are interleaved (re, im) doubles (C99 double
 * complex). Matrices are column-major with a leading dimension. Row index
 * i = m*Nm + T (testing MBF T on antenna m), column j = n*Nm + S (source MBF
 * S on antenna n). Coefficients c[T][S][p+P][q]. Self blocks: element
 * (T, S) of antenna a at self[a*self_stride + T + S*Nm].
 *
 * Every function is a direct transcription of its definition: no blocking,
 * no recurrences, no fusion. OpenMP (when compiled with it) only splits
 * independent outer loops (pairs, columns, right-hand sides); it never
 * changes the order of any floating-point sum.
 */
#include <complex.h>
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

static const double ORACLE_PI = 3.14159265358979323846;
static const double ORACLE_C0 = 299792458.0;  /* m/s */
/* mu0 / (4 pi) with the classical mu0 = 4 pi 1e-7 H/m. */
static const double ORACLE_MU0_OVER_4PI = 1e-7;

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* Wavenumber k = 2 pi f / c0 (rad/m). */
double oracle_wavenumber(double freq_hz) { return 2.0 * ORACLE_PI * freq_hz / ORACLE_C0; }

/* One off-diagonal block Z^{mn} (Eq. 1, 3, 4), written into Z at rows
 * m*Nm.., columns n*Nm... `dvar` = 1 uses d = 1/r, 2 uses d = 1/r^2.
 * `ff` (may be NULL) holds the Fourier coefficients g_p^{TS} of the
 * pattern product F_T^* . F_S of Eq. 1, index [T][S][p+P]. */
static void fill_block(int Nm, int P, int Q, double dx, double dy, double k, double omega,
                       const cplx* coef, const cplx* ff, int dvar, cplx* Zblk, long ldz) {
  const int np = 2 * P + 1, nq = Q + 1;
  const double r = hypot(dx, dy);
  const double alpha = atan2(dy, dx);
  const double d = (dvar == 2) ? 1.0 / (r * r) : 1.0 / r;
  /* e^{j p alpha} for each harmonic and d^q for each power (Eq. 3). */
  cplx* eh = (cplx*)malloc(sizeof(cplx) * np);
  double* dq = (double*)malloc(sizeof(double) * nq);
  for (int p = -P; p <= P; ++p) eh[p + P] = cexp(I * (double)p * alpha);
  for (int q = 0; q <= Q; ++q) dq[q] = pow(d, (double)q);
  const cplx phase = cexp(-I * k * r); /* e^{-jkr}, time convention e^{jwt} */
  for (int S = 0; S < Nm; ++S) {
    for (int T = 0; T < Nm; ++T) {
      const cplx* c = coef + ((size_t)T * Nm + S) * np * nq;
      cplx B = 0.0;
      for (int p = 0; p < np; ++p) {
        cplx poly = 0.0;
        for (int q = 0; q < nq; ++q) poly += c[p * nq + q] * dq[q];
        B += eh[p] * poly;
      }
      cplx z = B * phase; /* Eq. 4 without the far-field term */
      if (ff) {
        const cplx* g = ff + ((size_t)T * Nm + S) * np;
        cplx gpat = 0.0;
        for (int p = 0; p < np; ++p) gpat += g[p] * eh[p];
        /* Eq. 1: -j w mu0 g e^{-jkr} / (4 pi r) */
        z += -I * omega * ORACLE_MU0_OVER_4PI * gpat * phase / r;
      }
      Zblk[T + (size_t)S * ldz] = z;
    }
  }
  free(eh);
  free(dq);
}

/* Reduced MBF matrix (Eq. 4 for m != n, self blocks on the diagonal).
 * Returns 0, or -1 when two antennas coincide (r == 0). */
int oracle_fill(int Na, int Nm, int P, int Q, const double* pos, double freq_hz,
                const cplx* coef, const cplx* ff, int dvar,
                const cplx* self_blocks, long self_stride, cplx* Z, long ldz) {
  const double k = oracle_wavenumber(freq_hz);
  const double omega = 2.0 * ORACLE_PI * freq_hz;
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(| : bad)
  for (int n = 0; n < Na; ++n) {
    for (int m = 0; m < Na; ++m) {
      cplx* Zblk = Z + (size_t)m * Nm + (size_t)n * Nm * ldz;
      if (m == n) {
        const cplx* sb = self_blocks + (size_t)m * self_stride;
        for (int S = 0; S < Nm; ++S)
          for (int T = 0; T < Nm; ++T) Zblk[T + (size_t)S * ldz] = sb[T + (size_t)S * Nm];
        continue;
      }
      const double dx = pos[2 * m] - pos[2 * n];
      const double dy = pos[2 * m + 1] - pos[2 * n + 1];
      if (dx == 0.0 && dy == 0.0) {
        bad = 1;
        continue;
      }
      fill_block(Nm, P, Q, dx, dy, k, omega, coef, ff, dvar, Zblk, ldz);
    }
  }
  return bad ? -1 : 0;
}

/* LU factorisation with partial pivoting, PA = LU, in place (Golub & Van
 * Loan, Algorithm 3.4.1: right-looking outer-product Gaussian elimination).
 * The pivot of column k is the row of largest modulus |a_ik|, i >= k, first
 * index on ties. ipiv[k] is the (0-based) row swapped with row k. Returns
 * 0, or k+1 when column k has an exactly zero pivot. */
int oracle_lu(int N, cplx* A, long lda, int* ipiv) {
  int info = 0;
  for (int k = 0; k < N; ++k) {
    int piv = k;
    double best = cabs(A[k + (size_t)k * lda]);
    for (int i = k + 1; i < N; ++i) {
      double v = cabs(A[i + (size_t)k * lda]);
      if (v > best) {
        best = v;
        piv = i;
      }
    }
    ipiv[k] = piv;
    if (best == 0.0) {
      if (!info) info = k + 1;
      continue;
    }
    if (piv != k) {
      for (int j = 0; j < N; ++j) {
        cplx t = A[k + (size_t)j * lda];
        A[k + (size_t)j * lda] = A[piv + (size_t)j * lda];
        A[piv + (size_t)j * lda] = t;
      }
    }
    const cplx inv = 1.0 / A[k + (size_t)k * lda];
    for (int i = k + 1; i < N; ++i) A[i + (size_t)k * lda] *= inv;
#pragma omp parallel for schedule(static) if (N - k > 256)
    for (int j = k + 1; j < N; ++j) {
      const cplx u = A[k + (size_t)j * lda];
      if (u == 0.0) continue;
      cplx* aj = A + (size_t)j * lda;
      const cplx* l = A + (size_t)k * lda;
      for (int i = k + 1; i < N; ++i) aj[i] -= l[i] * u;
    }
  }
  return info;
}

/* Solve A X = B (trans 'N') or A^T X = B (trans 'T', plain transpose) with
 * the factors of oracle_lu. B (N x nrhs) is overwritten by X. */
void oracle_lu_solve(int N, const cplx* A, long lda, const int* ipiv, int nrhs, cplx* B, long ldb,
                     char trans) {
#pragma omp parallel for schedule(static)
  for (int c = 0; c < nrhs; ++c) {
    cplx* b = B + (size_t)c * ldb;
    if (trans == 'N' || trans == 'n') {
      /* b <- P b */
      for (int k = 0; k < N; ++k) {
        int p = ipiv[k];
        if (p != k) {
          cplx t = b[k];
          b[k] = b[p];
          b[p] = t;
        }
      }
      /* L y = b, unit lower, forward */
      for (int k = 0; k < N; ++k) {
        const cplx yk = b[k];
        for (int i = k + 1; i < N; ++i) b[i] -= A[i + (size_t)k * lda] * yk;
      }
      /* U x = y, upper, backward */
      for (int k = N - 1; k >= 0; --k) {
        b[k] /= A[k + (size_t)k * lda];
        const cplx xk = b[k];
        for (int i = 0; i < k; ++i) b[i] -= A[i + (size_t)k * lda] * xk;
      }
    } else {
      /* A = P^T L U, so A^T = U^T L^T P. U^T y = b (lower, forward). */
      for (int k = 0; k < N; ++k) {
        cplx s = b[k];
        for (int i = 0; i < k; ++i) s -= A[i + (size_t)k * lda] * b[i];
        b[k] = s / A[k + (size_t)k * lda];
      }
      /* L^T z = y (unit upper, backward). */
      for (int k = N - 1; k >= 0; --k) {
        cplx s = b[k];
        for (int i = k + 1; i < N; ++i) s -= A[i + (size_t)k * lda] * b[i];
        b[k] = s;
      }
      /* x = P^T z: undo the swaps in reverse order. */
      for (int k = N - 1; k >= 0; --k) {
        int p = ipiv[k];
        if (p != k) {
          cplx t = b[k];
          b[k] = b[p];
          b[p] = t;
        }
      }
    }
  }
}

/* Port response P = E^T X (Na x Na, column-major) where E selects row
 * m*Nm (MBF 0 of antenna m); returns J = sum |P_mn|^2. */
double oracle_port_objective(int Na, int Nm, const cplx* X, long ldx, cplx* Pout) {
  double J = 0.0;
  for (int n = 0; n < Na; ++n)
    for (int m = 0; m < Na; ++m) {
      cplx v = X[(size_t)m * Nm + (size_t)n * ldx];
      if (Pout) Pout[m + (size_t)n * Na] = v;
      J += creal(v) * creal(v) + cimag(v) * cimag(v);
    }
  return J;
}

/* Derivatives of one off-diagonal block with respect to r and alpha:
 *   dZ/dr     = e^{-jkr} sum_p e^{j p alpha} sum_q c_pq (-jk d^q + q d^{q-1} dd/dr)
 *   dZ/dalpha = e^{-jkr} sum_p (j p) e^{j p alpha} sum_q c_pq d^q
 * with dd/dr = -1/r^2 (d = 1/r) or -2/r^3 (d = 1/r^2). Far-field term not
 * included (it folds exactly into the q = 1 coefficients when d = 1/r). */
static void block_derivatives(int Nm, int P, int Q, double r, double alpha, double k,
                              const cplx* coef, int dvar, cplx* dZdr, cplx* dZda) {
  const int np = 2 * P + 1, nq = Q + 1;
  const double d = (dvar == 2) ? 1.0 / (r * r) : 1.0 / r;
  const double dd_dr = (dvar == 2) ? -2.0 / (r * r * r) : -1.0 / (r * r);
  const cplx phase = cexp(-I * k * r);
  for (int S = 0; S < Nm; ++S)
    for (int T = 0; T < Nm; ++T) {
      const cplx* c = coef + ((size_t)T * Nm + S) * np * nq;
      cplx gr = 0.0, ga = 0.0;
      for (int p = -P; p <= P; ++p) {
        const cplx e = cexp(I * (double)p * alpha);
        cplx polyr = 0.0, poly = 0.0;
        for (int q = 0; q <= Q; ++q) {
          const cplx cq = c[(p + P) * nq + q];
          const double dq = pow(d, (double)q);
          const double ddq = (q == 0) ? 0.0 : (double)q * pow(d, (double)(q - 1)) * dd_dr;
          polyr += cq * (-I * k * dq + ddq);
          poly += cq * dq;
        }
        gr += e * polyr;
        ga += I * (double)p * e * poly;
      }
      dZdr[T + (size_t)S * Nm] = phase * gr;
      dZda[T + (size_t)S * Nm] = phase * ga;
    }
}

/* Gradient of J with respect to the antenna positions, given the forward
 * solution X = Z^{-1} V and the adjoint Lambda = Z^{-T} E conj(P):
 *   G = Lambda X^T,  dJ/dx = -2 Re sum_ij G_ij dZ_ij/dx.
 * Each ordered pair (m, n), m != n, depends on Delta = x_m - x_n only:
 *   g = -2 Re sum_TS G^{mn}_TS (dZ/dr Delta/r + dZ/dalpha (-Dy, Dx)/r^2),
 *   grad[m] += g, grad[n] -= g.
 * grad is (Na, 2) row-major, overwritten. */
void oracle_grad_from_adjoint(int Na, int Nm, int P, int Q, const double* pos, double freq_hz,
                              const cplx* coef, int dvar, const cplx* Lam, const cplx* X, long ld,
                              int nrhs, double* grad) {
  const double k = oracle_wavenumber(freq_hz);
  const int Nm2 = Nm * Nm;
  memset(grad, 0, sizeof(double) * 2 * (size_t)Na);
  double* gpair = (double*)calloc((size_t)Na * Na * 2, sizeof(double));
#pragma omp parallel for schedule(dynamic, 4)
  for (int n = 0; n < Na; ++n) {
    cplx* dZdr = (cplx*)malloc(sizeof(cplx) * Nm2);
    cplx* dZda = (cplx*)malloc(sizeof(cplx) * Nm2);
    for (int m = 0; m < Na; ++m) {
      if (m == n) continue;
      const double dx = pos[2 * m] - pos[2 * n];
      const double dy = pos[2 * m + 1] - pos[2 * n + 1];
      const double r = hypot(dx, dy);
      const double alpha = atan2(dy, dx);
      block_derivatives(Nm, P, Q, r, alpha, k, coef, dvar, dZdr, dZda);
      double sx = 0.0, sy = 0.0;
      for (int S = 0; S < Nm; ++S)
        for (int T = 0; T < Nm; ++T) {
          const size_t i = (size_t)m * Nm + T, j = (size_t)n * Nm + S;
          cplx G = 0.0;
          for (int c = 0; c < nrhs; ++c) G += Lam[i + (size_t)c * ld] * X[j + (size_t)c * ld];
          const cplx a = dZdr[T + (size_t)S * Nm], b = dZda[T + (size_t)S * Nm];
          /* dZ/dDx = dZ/dr * Dx/r + dZ/dalpha * (-Dy/r^2); dZ/dDy likewise */
          const cplx zx = a * (dx / r) + b * (-dy / (r * r));
          const cplx zy = a * (dy / r) + b * (dx / (r * r));
          sx += -2.0 * creal(G * zx);
          sy += -2.0 * creal(G * zy);
        }
      gpair[2 * ((size_t)m * Na + n)] = sx;
      gpair[2 * ((size_t)m * Na + n) + 1] = sy;
    }
    free(dZdr);
    free(dZda);
  }
  /* grad[m] += g(m,n); grad[n] -= g(m,n), summed in a fixed order. */
  for (int m = 0; m < Na; ++m)
    for (int n = 0; n < Na; ++n) {
      if (m == n) continue;
      const double gx = gpair[2 * ((size_t)m * Na + n)], gy = gpair[2 * ((size_t)m * Na + n) + 1];
      grad[2 * m] += gx;
      grad[2 * m + 1] += gy;
      grad[2 * n] -= gx;
      grad[2 * n + 1] -= gy;
    }
  free(gpair);
}

/* Whole forward + adjoint for the port objective J = sum |(E^T Z^{-1} E)_mn|^2:
 * fill, LU, X = Z^{-1} E, P = E^T X, Lambda = Z^{-T} E conj(P), gradient.
 * Returns J through *J_out (may be NULL); grad may be NULL (forward only).
 * Returns 0, -1 on coincident antennas, or k+1 on a zero pivot. */
int oracle_port_objective_grad(int Na, int Nm, int P, int Q, const double* pos, double freq_hz,
                               const cplx* coef, int dvar, const cplx* self_blocks,
                               long self_stride, double* J_out, double* grad) {
  const int N = Na * Nm;
  cplx* Z = (cplx*)malloc(sizeof(cplx) * (size_t)N * N);
  cplx* X = (cplx*)calloc((size_t)N * Na, sizeof(cplx));
  int* ipiv = (int*)malloc(sizeof(int) * N);
  int rc = oracle_fill(Na, Nm, P, Q, pos, freq_hz, coef, NULL, dvar, self_blocks, self_stride, Z,
                       N);
  if (rc == 0) rc = oracle_lu(N, Z, N, ipiv);
  if (rc == 0) {
    for (int m = 0; m < Na; ++m) X[(size_t)m * Nm + (size_t)m * N] = 1.0;
    oracle_lu_solve(N, Z, N, ipiv, Na, X, N, 'N');
    cplx* Pm = (cplx*)malloc(sizeof(cplx) * (size_t)Na * Na);
    double J = oracle_port_objective(Na, Nm, X, N, Pm);
    if (J_out) *J_out = J;
    if (grad) {
      cplx* Lam = (cplx*)calloc((size_t)N * Na, sizeof(cplx));
      /* E conj(P): row m*Nm of column c holds conj(P_mc). */
      for (int c = 0; c < Na; ++c)
        for (int m = 0; m < Na; ++m) Lam[(size_t)m * Nm + (size_t)c * N] = conj(Pm[m + (size_t)c * Na]);
      oracle_lu_solve(N, Z, N, ipiv, Na, Lam, N, 'T');
      oracle_grad_from_adjoint(Na, Nm, P, Q, pos, freq_hz, coef, dvar, Lam, X, N, Na, grad);
      free(Lam);
    }
    free(Pm);
  }
  free(Z);
  free(X);
  free(ipiv);
  return rc;
}

/* ---- Section II-C, Eq. 5 and 6: embedded element patterns -----------------
 * The pattern of the array for the MBF coefficients c_ij (MBF j on antenna
 * i) is the double sum of Eq. 5,
 *   F(u) = sum_i sum_j c_ij F_j(u) e^{jk (u_x x_i + u_y y_i)},
 * evaluated here term by term as written (no factoring by the array
 * factor of Eq. 6). The embedded element pattern of port m is the pattern
 * of the currents for excitation at port m: c_ij = X[i*Nm + j, m].
 *   ux, uy   direction cosines of the D directions
 *   F        MBF patterns, index [comp][d][j] (comp 0: theta, 1: phi)
 *   E        output, index [comp][m][d] */
void oracle_eep(int Na, int Nm, const double* pos, double freq_hz, const cplx* X, long ldx,
                int nports, int D, const double* ux, const double* uy, const cplx* F, cplx* E) {
  const double k = oracle_wavenumber(freq_hz);
#pragma omp parallel for collapse(2) schedule(static)
  for (int m = 0; m < nports; ++m)
    for (int d = 0; d < D; ++d)
      for (int comp = 0; comp < 2; ++comp) {
        cplx s = 0.0;
        for (int i = 0; i < Na; ++i)
          for (int j = 0; j < Nm; ++j) {
            const cplx c = X[(size_t)i * Nm + j + (size_t)m * ldx];
            const cplx Fj = F[((size_t)comp * D + d) * Nm + j];
            const double ph = k * (ux[d] * pos[2 * i] + uy[d] * pos[2 * i + 1]);
            s += c * Fj * cexp(I * ph);
          }
        E[((size_t)comp * nports + m) * D + d] = s;
      }
}

/* Eq. 8: the error between two patterns in each direction,
 *   eps = sqrt(|E_theta - Eref_theta|^2 + |E_phi - Eref_phi|^2) / norm,
 * with the fields normalised by `norm` (the maximum of the isolated
 * antenna's pattern). E, Eref: [comp][n]; eps: [n]. */
void oracle_pattern_error(int n, const cplx* E, const cplx* Eref, double norm, double* eps) {
  for (int q = 0; q < n; ++q) {
    const double a = cabs(E[q] - Eref[q]), b = cabs(E[n + q] - Eref[n + q]);
    eps[q] = sqrt(a * a + b * b) / norm;
  }
}
