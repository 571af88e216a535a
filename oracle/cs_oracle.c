/*
 * Plain FP64 CPU oracle for the cuSten hot path (Gloster & O Naraigh, arXiv:1902.09931).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct statement of what the
 * GPU library computes.  Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark may build, load or call it; the GPU library never links or calls it and shares no
 * code, header, table or constant with it.
 *
 * Every routine is a direct loop over the definition it cites; nothing is blocked, fused or
 * reordered beyond what the definition states.  All arithmetic is IEEE binary64.
 *
 * Conventions (Sec. 2, Sec. 3, Sec. 5.2 of the paper):
 *   - A 2D field is stored row-major with x fastest: element (j, i) is at [j*nx + i]
 *     (the y-tiles of Sec. 2 are contiguous chunks of rows).
 *   - A stencil has `left`, `right` points in x and `top`, `bottom` points in y around (i, j).
 *     Weights are numbered from the top-left corner of the stencil box, left to right in i,
 *     then row by row in j (Sec. 5.2); the first row is j - top (smaller j, earlier in memory).
 *     So weight w[q*(left+right+1) + p] multiplies in[j - top + q][i - left + p].
 *   - Periodic boundaries wrap indices modulo the grid size (Sec. 3, "p").
 *   - Non-periodic boundaries leave every output cell whose stencil would leave the grid
 *     untouched (Sec. 3, "np"; Sec. 4.1): cells with i < left, i >= nx - right,
 *     j < top or j >= ny - bottom are not written.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-3)

enum { ORC_DIR_X = 0, ORC_DIR_Y = 1, ORC_DIR_XY = 2 };
enum { ORC_BC_NONPERIODIC = 0, ORC_BC_PERIODIC = 1 };
enum {
  ORC_FN_CENTRAL_D2X = 1,     /* Sec. 4.2: (u[i-1] - 2u[i] + u[i+1]) * coe[0], coe[0] = 1/dx^2 */
  ORC_FN_CH_NONLIN_LAP = 2,   /* Sec. 5.2: Laplacian of (C^3 - C), coe[0] = 1/h^2 */
  ORC_FN_CUBIC_MINUS_LAP = 3  /* c^3 - c - Laplacian(c), coe[0] = 1/h^2 */
};

static int64_t wrap(int64_t k, int64_t n) {
  int64_t r = k % n;
  return r < 0 ? r + n : r;
}

/* Sec. 2 / Sec. 3: weighted linear stencil, out = sum_k w_k * in(neighbour k). */
int orc_stencil2d(int64_t nx, int64_t ny, int dir, int bc, int left, int right, int top,
                  int bottom, const double* w, const double* in, double* out) {
  if (nx < 1 || ny < 1 || left < 0 || right < 0 || top < 0 || bottom < 0) return ORC_EINVAL;
  if (dir == ORC_DIR_X && (top != 0 || bottom != 0)) return ORC_EINVAL;
  if (dir == ORC_DIR_Y && (left != 0 || right != 0)) return ORC_EINVAL;
  if (dir < ORC_DIR_X || dir > ORC_DIR_XY || (bc != ORC_BC_PERIODIC && bc != ORC_BC_NONPERIODIC))
    return ORC_EINVAL;
  const int width = left + right + 1;
  const int height = top + bottom + 1;
  for (int64_t j = 0; j < ny; ++j) {
    for (int64_t i = 0; i < nx; ++i) {
      if (bc == ORC_BC_NONPERIODIC &&
          (i < left || i >= nx - right || j < top || j >= ny - bottom))
        continue; /* boundary cell: left untouched */
      double sum = 0.0;
      for (int q = 0; q < height; ++q) {
        for (int p = 0; p < width; ++p) {
          int64_t jj = j - top + q;
          int64_t ii = i - left + p;
          if (bc == ORC_BC_PERIODIC) {
            jj = wrap(jj, ny);
            ii = wrap(ii, nx);
          }
          sum += w[q * width + p] * in[jj * nx + ii];
        }
      }
      out[j * nx + i] = sum;
    }
  }
  return ORC_OK;
}

/* The stencil footprint each user function of Sec. 4.2 / Sec. 5.2 reads. */
static int fn_extent(int fn, int* left, int* right, int* top, int* bottom, int* ncoe) {
  switch (fn) {
    case ORC_FN_CENTRAL_D2X:
      *left = 1; *right = 1; *top = 0; *bottom = 0; *ncoe = 1;
      return ORC_OK;
    case ORC_FN_CH_NONLIN_LAP:
    case ORC_FN_CUBIC_MINUS_LAP:
      *left = 1; *right = 1; *top = 1; *bottom = 1; *ncoe = 1;
      return ORC_OK;
    default:
      return ORC_EINVAL;
  }
}

/* Value of the field at offset (dx, dy) from (i, j), periodic wrap when asked. */
static double at(const double* in, int64_t nx, int64_t ny, int bc, int64_t i, int64_t j,
                 int dx, int dy) {
  int64_t ii = i + dx, jj = j + dy;
  if (bc == ORC_BC_PERIODIC) {
    ii = wrap(ii, nx);
    jj = wrap(jj, ny);
  }
  return in[jj * nx + ii];
}

static double cubic_minus(double c) { return c * c * c - c; }

/* Sec. 4.2 / Sec. 5.2: user-function stencil.  The function sees the neighbourhood of (i, j)
 * and the coefficient array and returns the output value for (i, j). */
int orc_stencil2d_fn(int64_t nx, int64_t ny, int bc, int fn, const double* coe, int ncoe,
                     const double* in, double* out) {
  int left, right, top, bottom, need;
  if (fn_extent(fn, &left, &right, &top, &bottom, &need) != ORC_OK) return ORC_EINVAL;
  if (ncoe < need || nx < 1 || ny < 1) return ORC_EINVAL;
  if (bc != ORC_BC_PERIODIC && bc != ORC_BC_NONPERIODIC) return ORC_EINVAL;
  for (int64_t j = 0; j < ny; ++j) {
    for (int64_t i = 0; i < nx; ++i) {
      if (bc == ORC_BC_NONPERIODIC &&
          (i < left || i >= nx - right || j < top || j >= ny - bottom))
        continue;
      double v;
      if (fn == ORC_FN_CENTRAL_D2X) {
        /* Sec. 4.2: standard second-order central difference in x. */
        v = (at(in, nx, ny, bc, i, j, -1, 0) - 2.0 * at(in, nx, ny, bc, i, j, 0, 0) +
             at(in, nx, ny, bc, i, j, 1, 0)) * coe[0];
      } else {
        /* Five-point Laplacian (Eq. 5a in x plus the same in y, dx = dy) of N = C^3 - C
         * evaluated point by point (Sec. 5.2), or of C itself. */
        double lap_n = (cubic_minus(at(in, nx, ny, bc, i, j, -1, 0)) - 2.0 * cubic_minus(at(in, nx, ny, bc, i, j, 0, 0)) +
                        cubic_minus(at(in, nx, ny, bc, i, j, 1, 0))) * coe[0] +
                       (cubic_minus(at(in, nx, ny, bc, i, j, 0, -1)) - 2.0 * cubic_minus(at(in, nx, ny, bc, i, j, 0, 0)) +
                        cubic_minus(at(in, nx, ny, bc, i, j, 0, 1))) * coe[0];
        if (fn == ORC_FN_CH_NONLIN_LAP) {
          v = lap_n;
        } else {
          double c = at(in, nx, ny, bc, i, j, 0, 0);
          double lap_c = (at(in, nx, ny, bc, i, j, -1, 0) - 2.0 * c + at(in, nx, ny, bc, i, j, 1, 0)) * coe[0] +
                         (at(in, nx, ny, bc, i, j, 0, -1) - 2.0 * c + at(in, nx, ny, bc, i, j, 0, 1)) * coe[0];
          v = cubic_minus(c) - lap_c;
        }
      }
      out[j * nx + i] = v;
    }
  }
  return ORC_OK;
}

/* Batched 1D stencil (Abstract, Sec. 5.4: batches of 1D problems): the x-direction stencil of
 * Sec. 3 applied to each line m = [offsets[m], offsets[m+1]) of a packed buffer on its own,
 * wrapping at the line's own length when periodic. */
int orc_stencil1d_batch(int64_t num_lines, const int64_t* offsets, int bc, int left, int right,
                        const double* w, const double* in, double* out) {
  if (num_lines < 0 || left < 0 || right < 0) return ORC_EINVAL;
  if (bc != ORC_BC_PERIODIC && bc != ORC_BC_NONPERIODIC) return ORC_EINVAL;
  const int width = left + right + 1;
  for (int64_t m = 0; m < num_lines; ++m) {
    const int64_t start = offsets[m];
    const int64_t len = offsets[m + 1] - start;
    if (len < 0) return ORC_EINVAL;
    for (int64_t i = 0; i < len; ++i) {
      if (bc == ORC_BC_NONPERIODIC && (i < left || i >= len - right)) continue;
      double sum = 0.0;
      for (int p = 0; p < width; ++p) {
        int64_t ii = i - left + p;
        if (bc == ORC_BC_PERIODIC) ii = wrap(ii, len);
        sum += w[p] * in[start + ii];
      }
      out[start + i] = sum;
    }
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------------------------ */
/* Cyclic pentadiagonal solve (Sec. 5.1): (I + a P) x = b with P the periodic fourth-difference
 * matrix of Eq. 5b, P = circulant(1, -4, 6, -4, 1).  The periodic corners are treated as in the
 * cited pentadiagonal method: split M = A0 + U V^T, where A0 is the banded (non-cyclic) part and
 * U V^T holds the six corner entries, solve with A0 by banded Gaussian elimination, and correct
 * with the Sherman-Morrison-Woodbury formula
 *     x = y - Z (I + V^T Z)^{-1} V^T y,   y = A0^{-1} b,   Z = A0^{-1} U.                       */

/* Banded Gaussian elimination without pivoting on an SPD matrix of half-bandwidth 2, stored as
 * rows band[i][0..4] = columns i-2 .. i+2.  Factorises in place: the multipliers replace the
 * sub-diagonal entries. */
static void band_factor(int64_t n, double (*band)[5]) {
  for (int64_t k = 0; k < n; ++k) {
    for (int64_t r = k + 1; r <= k + 2 && r < n; ++r) {
      /* entry (r, k) sits at band[r][k - r + 2] */
      double l = band[r][k - r + 2] / band[k][2];
      band[r][k - r + 2] = l;
      for (int64_t c = k + 1; c <= k + 2 && c < n; ++c) band[r][c - r + 2] -= l * band[k][c - k + 2];
    }
  }
}

static void band_solve(int64_t n, double (*band)[5], double* x) {
  for (int64_t r = 0; r < n; ++r) /* forward: L y = b (unit lower) */
    for (int64_t k = (r >= 2 ? r - 2 : 0); k < r; ++k) x[r] -= band[r][k - r + 2] * x[k];
  for (int64_t r = n - 1; r >= 0; --r) { /* backward: U x = y */
    for (int64_t c = r + 1; c <= r + 2 && c < n; ++c) x[r] -= band[r][c - r + 2] * x[c];
    x[r] /= band[r][2];
  }
}

/* Dense Gaussian elimination with partial pivoting for the small capacitance system. */
static int dense_solve(int m, double* A, double* b) {
  for (int k = 0; k < m; ++k) {
    int piv = k;
    for (int r = k + 1; r < m; ++r)
      if (fabs(A[r * m + k]) > fabs(A[piv * m + k])) piv = r;
    if (A[piv * m + k] == 0.0) return ORC_EINVAL;
    if (piv != k) {
      for (int c = 0; c < m; ++c) {
        double t = A[k * m + c]; A[k * m + c] = A[piv * m + c]; A[piv * m + c] = t;
      }
      double t = b[k]; b[k] = b[piv]; b[piv] = t;
    }
    for (int r = k + 1; r < m; ++r) {
      double l = A[r * m + k] / A[k * m + k];
      for (int c = k; c < m; ++c) A[r * m + c] -= l * A[k * m + c];
      b[r] -= l * b[k];
    }
  }
  for (int r = m - 1; r >= 0; --r) {
    for (int c = r + 1; c < m; ++c) b[r] -= A[r * m + c] * b[c];
    b[r] /= A[r * m + r];
  }
  return ORC_OK;
}

/* Solves num_rhs systems (I + a P) x = b, each b a contiguous vector of length n (n >= 5). */
int orc_cyclic_penta_solve(int64_t n, double a, int64_t num_rhs, const double* b, double* x) {
  if (n < 5 || num_rhs < 0) return ORC_EINVAL;
  double (*band)[5] = malloc(sizeof(double[5]) * n);
  double* z = malloc(sizeof(double) * 4 * n); /* Z = A0^{-1} U, column-major n x 4 */
  if (!band || !z) { free(band); free(z); return ORC_ENOMEM; }
  /* A0: rows of I + a * (1, -4, 6, -4, 1) without the wrap-around entries. */
  for (int64_t i = 0; i < n; ++i) {
    const double row[5] = {a, -4.0 * a, 1.0 + 6.0 * a, -4.0 * a, a};
    for (int d = 0; d < 5; ++d) {
      int64_t c = i + d - 2;
      band[i][d] = (c >= 0 && c < n) ? row[d] : 0.0;
    }
  }
  band_factor(n, band);
  /* Corner entries of M that A0 lacks, in the index set K = {0, 1, n-2, n-1}:
   *   M[0][n-2] = a, M[0][n-1] = -4a, M[1][n-1] = a,
   *   M[n-2][0] = a, M[n-1][0] = -4a, M[n-1][1] = a.
   * U = columns e_0, e_1, e_{n-2}, e_{n-1}; V^T = the corner block acting on K, so that
   * (U V^T)[K[r]][K[c]] = Ck[r][c].                                                         */
  const int64_t K[4] = {0, 1, n - 2, n - 1};
  double Ck[16] = {0};
  Ck[0 * 4 + 2] = a;          /* row 0, col n-2 */
  Ck[0 * 4 + 3] = -4.0 * a;   /* row 0, col n-1 */
  Ck[1 * 4 + 3] = a;          /* row 1, col n-1 */
  Ck[2 * 4 + 0] = a;          /* row n-2, col 0 */
  Ck[3 * 4 + 0] = -4.0 * a;   /* row n-1, col 0 */
  Ck[3 * 4 + 1] = a;          /* row n-1, col 1 */
  for (int r = 0; r < 4; ++r) {
    double* zr = z + r * n;
    memset(zr, 0, sizeof(double) * n);
    zr[K[r]] = 1.0;
    band_solve(n, band, zr);
  }
  /* Capacitance matrix S = I + V^T Z, with (V^T Z)[r][c] = sum_s Ck[r][s] * Z[K[s]][c]. */
  double S[16];
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) {
      double s = (r == c) ? 1.0 : 0.0;
      for (int t = 0; t < 4; ++t) s += Ck[r * 4 + t] * z[c * n + K[t]];
      S[r * 4 + c] = s;
    }
  int rc = ORC_OK;
  for (int64_t m = 0; m < num_rhs && rc == ORC_OK; ++m) {
    double* xm = x + m * n;
    memmove(xm, b + m * n, sizeof(double) * n);
    band_solve(n, band, xm); /* y = A0^{-1} b */
    double t[4], Sw[16];
    for (int r = 0; r < 4; ++r) { /* V^T y */
      t[r] = 0.0;
      for (int s = 0; s < 4; ++s) t[r] += Ck[r * 4 + s] * xm[K[s]];
    }
    memcpy(Sw, S, sizeof S);
    rc = dense_solve(4, Sw, t); /* t = S^{-1} V^T y */
    for (int64_t i = 0; i < n; ++i)
      for (int c = 0; c < 4; ++c) xm[i] -= z[c * n + i] * t[c];
  }
  free(band);
  free(z);
  return rc;
}

/* ------------------------------------------------------------------------------------------ */
/* Cahn-Hilliard ADI step (Sec. 5, Eq. ch_adi), periodic on (0, 2 pi)^2 with n x n points,
 * h = dx = dy = 2 pi / n.
 *   Cbar = 2 C^n - C^{n-1}                                   (extrapolated level n+1)
 *   RHS  = -(2/3)(C^n - C^{n-1}) - (2/3) D gamma dt lap4 Cbar + (2/3) D dt lap2 (C^3 - C)^n
 *   L_x w = RHS,  L_y v = w,  C^{n+1} = Cbar + v,  L = I + (2/3) D gamma dt d^4
 * lap2 = dxx + dyy (Eq. 5a), lap4 = dxxxx + 2 dxxyy + dyyyy (Eq. 5b and the cross stencil of
 * Fig. 1).  The coefficient D gamma on the lap4 term is the reading that makes the scheme
 * consistent with L_x (the printed equation omits it).                                       */

static double d2x(const double* f, int64_t n, int64_t i, int64_t j, double h2) {
  return (f[j * n + wrap(i - 1, n)] - 2.0 * f[j * n + i] + f[j * n + wrap(i + 1, n)]) / h2;
}
static double d2y(const double* f, int64_t n, int64_t i, int64_t j, double h2) {
  return (f[wrap(j - 1, n) * n + i] - 2.0 * f[j * n + i] + f[wrap(j + 1, n) * n + i]) / h2;
}
static double d4x(const double* f, int64_t n, int64_t i, int64_t j, double h4) {
  return (f[j * n + wrap(i - 2, n)] - 4.0 * f[j * n + wrap(i - 1, n)] + 6.0 * f[j * n + i] -
          4.0 * f[j * n + wrap(i + 1, n)] + f[j * n + wrap(i + 2, n)]) / h4;
}
static double d4y(const double* f, int64_t n, int64_t i, int64_t j, double h4) {
  return (f[wrap(j - 2, n) * n + i] - 4.0 * f[wrap(j - 1, n) * n + i] + 6.0 * f[j * n + i] -
          4.0 * f[wrap(j + 1, n) * n + i] + f[wrap(j + 2, n) * n + i]) / h4;
}
/* Fig. 1: second-order cross derivative d^4/dx^2dy^2 = (1,-2,1) (x) (1,-2,1) / h^4. */
static double d2x2y(const double* f, int64_t n, int64_t i, int64_t j, double h4) {
  const double c[3] = {1.0, -2.0, 1.0};
  double s = 0.0;
  for (int q = 0; q < 3; ++q)
    for (int p = 0; p < 3; ++p) s += c[q] * c[p] * f[wrap(j - 1 + q, n) * n + wrap(i - 1 + p, n)];
  return s / h4;
}

/* Computes the right-hand side of the x-sweep; exposed so tests can scale per-step errors. */
int orc_ch_rhs(int64_t n, double D, double gamma, double dt, const double* c_prev,
               const double* c_cur, double* rhs) {
  if (n < 5) return ORC_EINVAL;
  const double h = 2.0 * M_PI / (double)n;
  const double h2 = h * h, h4 = h2 * h2;
  const int64_t nn = n * n;
  double* cbar = malloc(sizeof(double) * nn);
  double* nl = malloc(sizeof(double) * nn);
  if (!cbar || !nl) { free(cbar); free(nl); return ORC_ENOMEM; }
  for (int64_t k = 0; k < nn; ++k) {
    cbar[k] = 2.0 * c_cur[k] - c_prev[k];
    nl[k] = c_cur[k] * c_cur[k] * c_cur[k] - c_cur[k];
  }
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) {
      double lap4 = d4x(cbar, n, i, j, h4) + 2.0 * d2x2y(cbar, n, i, j, h4) + d4y(cbar, n, i, j, h4);
      double lap2 = d2x(nl, n, i, j, h2) + d2y(nl, n, i, j, h2);
      rhs[j * n + i] = -(2.0 / 3.0) * (c_cur[j * n + i] - c_prev[j * n + i]) -
                       (2.0 / 3.0) * D * gamma * dt * lap4 + (2.0 / 3.0) * D * dt * lap2;
    }
  free(cbar);
  free(nl);
  return ORC_OK;
}

int orc_ch_step(int64_t n, double D, double gamma, double dt, const double* c_prev,
                const double* c_cur, double* c_next) {
  if (n < 5) return ORC_EINVAL;
  const double h = 2.0 * M_PI / (double)n;
  const double a = (2.0 / 3.0) * D * gamma * dt / (h * h * h * h);
  const int64_t nn = n * n;
  double* rhs = malloc(sizeof(double) * nn);
  double* w = malloc(sizeof(double) * nn);
  double* col = malloc(sizeof(double) * 2 * n);
  if (!rhs || !w || !col) { free(rhs); free(w); free(col); return ORC_ENOMEM; }
  int rc = orc_ch_rhs(n, D, gamma, dt, c_prev, c_cur, rhs);
  /* L_x w = RHS: every row is a contiguous line. */
  if (rc == ORC_OK) rc = orc_cyclic_penta_solve(n, a, n, rhs, w);
  /* L_y v = w: every column, gathered into a contiguous line. */
  for (int64_t i = 0; i < n && rc == ORC_OK; ++i) {
    for (int64_t j = 0; j < n; ++j) col[j] = w[j * n + i];
    rc = orc_cyclic_penta_solve(n, a, 1, col, col + n);
    for (int64_t j = 0; j < n; ++j) {
      double cbar = 2.0 * c_cur[j * n + i] - c_prev[j * n + i];
      c_next[j * n + i] = cbar + col[n + j];
    }
  }
  free(rhs);
  free(w);
  free(col);
  return rc;
}

/* Mass  M = h^2 sum C  (the integral of C over the periodic box). */
double orc_ch_mass(int64_t n, const double* c) {
  const double h = 2.0 * M_PI / (double)n;
  double s = 0.0;
  for (int64_t k = 0; k < n * n; ++k) s += c[k];
  return h * h * s;
}

/* Free energy F[C] of Sec. 5 (Eq. 1), the integral of 1/4 (C^2-1)^2 + gamma/2 |grad C|^2,
 * with the gradient taken by periodic forward differences and the integral by the rectangle
 * rule on the periodic grid. */
double orc_ch_energy(int64_t n, double gamma, const double* c) {
  const double h = 2.0 * M_PI / (double)n;
  double s = 0.0;
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) {
      double v = c[j * n + i];
      double gx = (c[j * n + wrap(i + 1, n)] - v) / h;
      double gy = (c[wrap(j + 1, n) * n + i] - v) / h;
      s += 0.25 * (v * v - 1.0) * (v * v - 1.0) + 0.5 * gamma * (gx * gx + gy * gy);
    }
  return h * h * s;
}

/* The time loop of Sec. 5.1: C^{-1} := C^0 on the first step, then nsteps ADI steps.
 * Writes the final C into c_out and, when non-null, the mass and energy after every step. */
int orc_ch_run(int64_t n, double D, double gamma, double dt, int64_t nsteps, const double* c0,
               double* c_out, double* mass, double* energy) {
  if (n < 5 || nsteps < 0) return ORC_EINVAL;
  const int64_t nn = n * n;
  double* prev = malloc(sizeof(double) * nn);
  double* cur = malloc(sizeof(double) * nn);
  double* next = malloc(sizeof(double) * nn);
  if (!prev || !cur || !next) { free(prev); free(cur); free(next); return ORC_ENOMEM; }
  memcpy(prev, c0, sizeof(double) * nn);
  memcpy(cur, c0, sizeof(double) * nn);
  int rc = ORC_OK;
  for (int64_t s = 0; s < nsteps && rc == ORC_OK; ++s) {
    rc = orc_ch_step(n, D, gamma, dt, prev, cur, next);
    double* t = prev; prev = cur; cur = next; next = t;
    if (mass) mass[s] = orc_ch_mass(n, cur);
    if (energy) energy[s] = orc_ch_energy(n, gamma, cur);
  }
  memcpy(c_out, cur, sizeof(double) * nn);
  free(prev);
  free(cur);
  free(next);
  return rc;
}
