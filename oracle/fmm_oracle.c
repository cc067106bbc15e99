/*
 * fmm_oracle.c -- plain, slow, CPU reference of the compressed-Taylor FMM of
 * Fernando & Kloeckner, "Automatic Synthesis of Low-Complexity Translation
 * Operators for the Fast Multipole Method" (arXiv 2305.17867).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py load this library.  It shares no
 * code, header, table or generator with the CUDA path, and the CUDA path
 * never loads it.
 *
 * Arithmetic is IEEE double throughout, except the radial derivative sums
 * (Sec. 4.4), which are carried in long double to keep the reference well
 * below the 1e-12 parity bar at derivative orders up to 2p = 32.
 * Compile without -ffast-math: the sums below are meant to run as written.
 *
 * Readings of the paper used here:
 *  R1  N(p) = C(p+d, d): the number of multi-indices of total order <= p
 *      (the binomial printed in eq. (np-count) drops the "+d").
 *  R2  Multipole basis: derivatives of G in its argument evaluated at x - c,
 *      coefficients (c - y)^q / q!  (Sec. 2, eq. (mpole), Sec. 3.4).
 *  R3  The graded order nu (Def. 1) is: total degree first, then the LAST
 *      coordinate ascending (it varies slowest, Lemma 5 with k = d), then the
 *      next-to-last ascending, and so on.  Hence c*e_d is the last element of
 *      M(c), and for a PDE with a_{c e_d} != 0 the stored set is
 *      j = { m in M(p) : m_d < c }.
 *  R4  Local expansions are stored as un-normalised derivatives of the
 *      potential at the centre (eq. (stored_local_coeffs)); the 1/m! is
 *      applied at evaluation (eq. (compressed-local-form)) and in L2L.
 *  R5  Kernels: 2D Laplace G = log r; 3D Laplace G = 1/(4 pi r); 3D Yukawa
 *      G = exp(-lambda r)/r with PDE Laplacian - lambda^2; 3D biharmonic
 *      G = r with PDE Laplacian^2; 2D biharmonic G = r^2 log r.
 *  R6  Pairs with x == y exactly are left out of every direct sum.
 *  R7  Uniform tree: leaf depth L, root = level 0; M2L at levels 2..L over
 *      the interaction list (List 2): children of the parent's neighbours
 *      (parent included) that are not adjacent to the box.
 *  R15 Adaptive tree: a box splits while it holds more than max_leaf points
 *      (sources plus targets) and is above max_depth; empty children are not
 *      created; lists U, V, W, X as defined above or_fmm_adaptive (the paper
 *      only cites the adaptive FMM it builds on).
 */
#define _GNU_SOURCE
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXD 3

/* Helmholtz G = e^{i kappa r}/r (PDE Laplacian + kappa^2) is carried as its
 * real and imaginary parts, cos(kappa r)/r and sin(kappa r)/r: both satisfy
 * the same real PDE, so with real weights the multipoles, their compression
 * and M2M are real and shared, and every later stage is linear in G.  The
 * parameter lam is kappa for these two kernels. */
enum { OR_LAPLACE = 0, OR_YUKAWA = 1, OR_BIHARMONIC = 2, OR_HELM_RE = 3, OR_HELM_IM = 4 };

enum {
  OR_OK = 0,
  OR_ERR_ARG = -1,
  OR_ERR_UNSUPPORTED = -2,
  OR_ERR_NOMEM = -4,
  OR_ERR_DOMAIN = -6
};

/* ------------------------------------------------------------------------ */
/* Multi-index algebra: Sec. 2 (M(p), N(p)) and Def. 1 (graded order nu).    */
/* ------------------------------------------------------------------------ */

static long or_binom(int n, int k) {
  if (k < 0 || n < 0 || k > n) return 0;
  long r = 1;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}

/* N(p) = |M(p)| = C(p+d, d)  (reading R1). */
int or_num_terms(int d, int p) { return p < 0 ? 0 : (int)or_binom(p + d, d); }

/* Enumerate M(p) in the order nu of reading R3; out has N(p)*d entries. */
void or_multi_indices(int d, int p, int* out) {
  int idx = 0;
  for (int n = 0; n <= p; ++n) {
    if (d == 1) {
      out[idx++] = n;
    } else if (d == 2) {
      for (int y = 0; y <= n; ++y) {
        out[2 * idx] = n - y;
        out[2 * idx + 1] = y;
        ++idx;
      }
    } else {
      for (int z = 0; z <= n; ++z)
        for (int y = 0; y <= n - z; ++y) {
          out[3 * idx] = n - z - y;
          out[3 * idx + 1] = y;
          out[3 * idx + 2] = z;
          ++idx;
        }
    }
  }
}

/* nu^{-1}: position of multi-index m in the order of reading R3. */
int or_mi_index(int d, const int* m) {
  int n = 0;
  for (int k = 0; k < d; ++k) n += m[k];
  int pos = or_num_terms(d, n - 1);
  if (d == 2) pos += m[1];
  if (d == 3) {
    for (int z = 0; z < m[2]; ++z) pos += n - z + 1;
    pos += m[1];
  }
  return pos;
}

static double or_mi_factorial(int d, const int* m) {
  double f = 1.0;
  for (int k = 0; k < d; ++k)
    for (int i = 2; i <= m[k]; ++i) f *= (double)i;
  return f;
}

/* ------------------------------------------------------------------------ */
/* The PDE operator L = sum_{m in M(c)} a_m d^m  (eq. (define_pde_op)).      */
/* Coefficients are returned densely over M(c) in nu order.                  */
/* ------------------------------------------------------------------------ */

/* Returns the PDE order c and fills acoef[N(c)] (caller gives >= N(4)). */
int or_pde_for_kernel(int kernel, int d, double lam, double* acoef) {
  int m[OR_MAXD];
  if (kernel == OR_LAPLACE || kernel == OR_YUKAWA || kernel == OR_HELM_RE ||
      kernel == OR_HELM_IM) {
    int c = 2;
    int nc = or_num_terms(d, c);
    for (int i = 0; i < nc; ++i) acoef[i] = 0.0;
    for (int k = 0; k < d; ++k) {
      for (int i = 0; i < d; ++i) m[i] = (i == k) ? 2 : 0;
      acoef[or_mi_index(d, m)] = 1.0;
    }
    if (kernel != OR_LAPLACE) {
      /* Yukawa: Laplacian - lambda^2; Helmholtz: Laplacian + kappa^2 */
      for (int i = 0; i < d; ++i) m[i] = 0;
      acoef[or_mi_index(d, m)] = kernel == OR_YUKAWA ? -lam * lam : lam * lam;
    }
    return c;
  }
  if (kernel == OR_BIHARMONIC) {
    /* (sum_k d_k^2)^2 = sum_k d_k^4 + 2 sum_{k<l} d_k^2 d_l^2 */
    int c = 4;
    int nc = or_num_terms(d, c);
    for (int i = 0; i < nc; ++i) acoef[i] = 0.0;
    for (int k = 0; k < d; ++k)
      for (int l = 0; l < d; ++l) {
        for (int i = 0; i < d; ++i) m[i] = 0;
        m[k] += 2;
        m[l] += 2;
        acoef[or_mi_index(d, m)] += 1.0;
      }
    return c;
  }
  return -1;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.1: the PDE matrix P (eqs. (coeff-shift), (define_P)), the pivot    */
/* map h (eq. (define_h)), the sets jbar (eq. (define_bar_j)) and j, and the */
/* decompression operator M with M[j,:] = I, M[jbar,:] = -P[:,jbar]^{-1}     */
/* P[:,j] (eq. (decompression)).  M is built densely, literally from its     */
/* definition, by forward substitution on the lower-triangular P[:,jbar]     */
/* (Lemma 3).                                                                 */
/* ------------------------------------------------------------------------ */

typedef struct {
  int d, p, c;
  int nfull;      /* N(p) */
  int nj;         /* |j| */
  int* mi;        /* nfull*d multi-indices in nu order */
  int* j;         /* nj positions (into nu order) of the stored set */
  int* is_stored; /* nfull flags */
  double* M;      /* nfull x nj, row-major */
} or_expansion;

void or_expansion_free(or_expansion* e) {
  if (!e) return;
  free(e->mi);
  free(e->j);
  free(e->is_stored);
  free(e->M);
  free(e);
}

/* b_{n,m} of eq. (coeff-shift); acoef is dense over M(c). */
static double or_b(int d, int c, const double* acoef, const int* n, const int* m) {
  int diff[OR_MAXD], s = 0;
  for (int k = 0; k < d; ++k) {
    diff[k] = m[k] - n[k];
    if (diff[k] < 0) return 0.0;
    s += diff[k];
  }
  if (s > c) return 0.0;
  return acoef[or_mi_index(d, diff)];
}

/* Build the expansion for order p and PDE (order c, coefficients acoef over
 * M(c)).  compressed == 0 gives the plain Taylor expansion (j = all, M = I). */
or_expansion* or_expansion_new(int d, int p, int c, const double* acoef,
                               int compressed) {
  or_expansion* e = (or_expansion*)calloc(1, sizeof(or_expansion));
  if (!e) return NULL;
  e->d = d;
  e->p = p;
  e->c = c;
  e->nfull = or_num_terms(d, p);
  e->mi = (int*)malloc(sizeof(int) * e->nfull * d);
  e->is_stored = (int*)calloc(e->nfull, sizeof(int));
  or_multi_indices(d, p, e->mi);
  int nrow = compressed ? or_num_terms(d, p - c) : 0; /* N(p-c) rows of P */
  int* h = (int*)malloc(sizeof(int) * (nrow > 0 ? nrow : 1));
  double* P = NULL;
  if (nrow > 0) {
    P = (double*)calloc((size_t)nrow * e->nfull, sizeof(double));
    for (int i = 0; i < nrow; ++i) {
      h[i] = -1;
      for (int l = 0; l < e->nfull; ++l) {
        double b = or_b(d, c, acoef, e->mi + i * d, e->mi + l * d);
        P[(size_t)i * e->nfull + l] = b;
        if (b != 0.0) h[i] = l; /* last nonzero column, eq. (define_h) */
      }
    }
  }
  for (int l = 0; l < e->nfull; ++l) e->is_stored[l] = 1;
  for (int i = 0; i < nrow; ++i) e->is_stored[h[i]] = 0;
  e->nj = 0;
  for (int l = 0; l < e->nfull; ++l) e->nj += e->is_stored[l];
  e->j = (int*)malloc(sizeof(int) * e->nj);
  {
    int t = 0;
    for (int l = 0; l < e->nfull; ++l)
      if (e->is_stored[l]) e->j[t++] = l;
  }
  e->M = (double*)calloc((size_t)e->nfull * e->nj, sizeof(double));
  for (int t = 0; t < e->nj; ++t) e->M[(size_t)e->j[t] * e->nj + t] = 1.0;
  if (nrow > 0) {
    /* X = -P[:,jbar]^{-1} P[:,j], row by row (P[:,jbar] lower triangular). */
    double* X = (double*)calloc((size_t)nrow * e->nj, sizeof(double));
    for (int i = 0; i < nrow; ++i) {
      double* xi = X + (size_t)i * e->nj;
      for (int t = 0; t < e->nj; ++t) xi[t] = -P[(size_t)i * e->nfull + e->j[t]];
      for (int i2 = 0; i2 < i; ++i2) {
        double pik = P[(size_t)i * e->nfull + h[i2]];
        if (pik == 0.0) continue;
        const double* x2 = X + (size_t)i2 * e->nj;
        for (int t = 0; t < e->nj; ++t) xi[t] -= pik * x2[t];
      }
      double diag = P[(size_t)i * e->nfull + h[i]];
      for (int t = 0; t < e->nj; ++t) xi[t] /= diag;
      memcpy(e->M + (size_t)h[i] * e->nj, xi, sizeof(double) * e->nj);
    }
    free(X);
  }
  free(P);
  free(h);
  return e;
}

int or_expansion_info(const or_expansion* e, int* nfull, int* nj) {
  *nfull = e->nfull;
  *nj = e->nj;
  return e->c;
}
void or_expansion_stored(const or_expansion* e, int* j) {
  memcpy(j, e->j, sizeof(int) * e->nj);
}
void or_expansion_matrix(const or_expansion* e, double* M) {
  memcpy(M, e->M, sizeof(double) * (size_t)e->nfull * e->nj);
}

/* D = M s  (decompression, eq. (decompression)); s has nj, D has nfull. */
void or_decompress(const or_expansion* e, const double* s, double* D) {
  for (int l = 0; l < e->nfull; ++l) {
    double acc = 0.0;
    const double* row = e->M + (size_t)l * e->nj;
    for (int t = 0; t < e->nj; ++t) acc += row[t] * s[t];
    D[l] = acc;
  }
}

/* beta = M^T alpha  (compression, eq. (define_beta_multipole)). */
void or_compress(const or_expansion* e, const double* alpha, double* beta) {
  for (int t = 0; t < e->nj; ++t) beta[t] = 0.0;
  for (int l = 0; l < e->nfull; ++l) {
    const double* row = e->M + (size_t)l * e->nj;
    double a = alpha[l];
    if (a == 0.0) continue;
    for (int t = 0; t < e->nj; ++t) beta[t] += row[t] * a;
  }
}

/* ------------------------------------------------------------------------ */
/* Derivatives of G (Sec. 4.4).  For a radially symmetric G(x) = F(s) with   */
/* s = |x|^2/2, the radial derivatives F^(n)(s) = ((1/r) d/dr)^n G (eq.      */
/* (tausch-dist-derivatives)) give every Cartesian derivative through the    */
/* chain rule in closed form:                                                */
/*   d^k G = sum_{0 <= 2 mu <= k} prod_i k_i! / (mu_i! (k_i-2mu_i)! 2^mu_i)  */
/*           x^(k-2mu) F^(|k|-|mu|)(s).                                       */
/* (In one variable, d^n/dx^n F(x^2/2) has exactly these Hermite-type terms; */
/* the variables separate because s is a sum of per-coordinate squares.)     */
/* ------------------------------------------------------------------------ */

/* Quad precision for the derivative sums: binary128 on both x86-64 (via
 * libquadmath) and aarch64 (where long double is binary128). */
#if defined(__x86_64__) && defined(__SIZEOF_FLOAT128__)
#include <quadmath.h>
typedef __float128 ld;
#define LD_LOG logq
#define LD_EXP expq
#define LD_SQRT sqrtq
#define LD_COS cosq
#define LD_SIN sinq
#define LDC(x) x##Q
#else
typedef long double ld;
#define LD_LOG logl
#define LD_EXP expl
#define LD_SQRT sqrtl
#define LD_COS cosl
#define LD_SIN sinl
#define LDC(x) x##L
#endif

/* F^(n)(s) for n = 0..nmax at radius r. */
static void or_radial(int kernel, int d, double lam, ld r, int nmax, ld* F) {
  const ld pi = LDC(3.141592653589793238462643383279502884);
  if (kernel == OR_LAPLACE && d == 3) {
    /* G = 1/(4 pi r): ((1/r)d/dr)^n r^-1 = (-1)^n (2n-1)!! r^-(2n+1) */
    ld rinv = LDC(1.0) / r, rinv2 = rinv * rinv, v = rinv / (LDC(4.0) * pi);
    for (int n = 0; n <= nmax; ++n) {
      F[n] = v;
      v *= -(ld)(2 * n + 1) * rinv2;
    }
  } else if (kernel == OR_LAPLACE && d == 2) {
    /* G = log r = (1/2) log(2s): F^(n) = (-1)^(n-1) (n-1)! / (2 s^n) */
    ld s = LDC(0.5) * r * r;
    F[0] = LD_LOG(r);
    ld v = LDC(1.0) / (LDC(2.0) * s);
    for (int n = 1; n <= nmax; ++n) {
      F[n] = v;
      v *= -(ld)n / s;
    }
  } else if (kernel == OR_YUKAWA && d == 3) {
    /* G = exp(-lam r)/r; F^(n) = exp(-lam r) sum_k c[n][k] r^-k, and
       (1/r)d/dr [e^{-lam r} r^-k] = e^{-lam r} (-lam r^-(k+1) - k r^-(k+2)). */
    int kmax = 2 * nmax + 2;
    ld* cc = (ld*)calloc((size_t)(kmax + 1), sizeof(ld));
    ld* cn = (ld*)calloc((size_t)(kmax + 1), sizeof(ld));
    cc[1] = LDC(1.0);
    ld e = LD_EXP(-(ld)lam * r), rinv = LDC(1.0) / r;
    for (int n = 0; n <= nmax; ++n) {
      ld acc = LDC(0.0), rp = LDC(1.0);
      for (int k = 0; k <= kmax; ++k) {
        acc += cc[k] * rp;
        rp *= rinv;
      }
      F[n] = e * acc;
      for (int k = 0; k <= kmax; ++k) cn[k] = LDC(0.0);
      for (int k = 0; k + 2 <= kmax; ++k) {
        if (cc[k] == LDC(0.0)) continue;
        cn[k + 1] += -(ld)lam * cc[k];
        cn[k + 2] += -(ld)k * cc[k];
      }
      for (int k = 0; k <= kmax; ++k) cc[k] = cn[k];
    }
    free(cc);
    free(cn);
  } else if ((kernel == OR_HELM_RE || kernel == OR_HELM_IM) && d == 3) {
    /* G = e^{i kappa r}/r, F^(n) = e^{i kappa r} sum_k c[n][k] r^-k with
       complex c: (1/r)d/dr [e^{i kappa r} r^-k] = e^{i kappa r} (i kappa r^-(k+1)
       - k r^-(k+2)); the real or the imaginary part is kept. */
    int kmax = 2 * nmax + 2;
    ld* cr = (ld*)calloc((size_t)(kmax + 1), sizeof(ld));
    ld* ci = (ld*)calloc((size_t)(kmax + 1), sizeof(ld));
    ld* nr = (ld*)calloc((size_t)(kmax + 1), sizeof(ld));
    ld* ni = (ld*)calloc((size_t)(kmax + 1), sizeof(ld));
    cr[1] = LDC(1.0);
    const ld kap = (ld)lam, rinv = LDC(1.0) / r;
    const ld er = LD_COS(kap * r), ei = LD_SIN(kap * r);
    for (int n = 0; n <= nmax; ++n) {
      ld ar = LDC(0.0), ai = LDC(0.0), rp = LDC(1.0);
      for (int k = 0; k <= kmax; ++k) {
        ar += cr[k] * rp;
        ai += ci[k] * rp;
        rp *= rinv;
      }
      F[n] = kernel == OR_HELM_RE ? er * ar - ei * ai : er * ai + ei * ar;
      for (int k = 0; k <= kmax; ++k) nr[k] = ni[k] = LDC(0.0);
      for (int k = 0; k + 2 <= kmax; ++k) {
        /* (i kappa) (cr + i ci) = -kappa ci + i kappa cr */
        nr[k + 1] += -kap * ci[k];
        ni[k + 1] += kap * cr[k];
        nr[k + 2] += -(ld)k * cr[k];
        ni[k + 2] += -(ld)k * ci[k];
      }
      for (int k = 0; k <= kmax; ++k) {
        cr[k] = nr[k];
        ci[k] = ni[k];
      }
    }
    free(cr);
    free(ci);
    free(nr);
    free(ni);
  } else if (kernel == OR_BIHARMONIC && d == 3) {
    /* G = r: F = r, then ((1/r)d/dr)^(n-1) r^-1 = (-1)^(n-1) (2n-3)!! r^-(2n-1) */
    ld rinv = LDC(1.0) / r, rinv2 = rinv * rinv;
    F[0] = r;
    ld v = rinv;
    for (int n = 1; n <= nmax; ++n) {
      F[n] = v;
      v *= -(ld)(2 * n - 1) * rinv2;
    }
  } else if (kernel == OR_BIHARMONIC && d == 2) {
    /* G = r^2 log r = s log(2s): F' = log(2s) + 1, F^(n) = (-1)^n (n-2)!/s^(n-1) */
    ld s = LDC(0.5) * r * r;
    F[0] = r * r * LD_LOG(r);
    if (nmax >= 1) F[1] = LDC(2.0) * LD_LOG(r) + LDC(1.0);
    ld v = LDC(1.0) / s;
    for (int n = 2; n <= nmax; ++n) {
      F[n] = v;
      v *= -(ld)(n - 1) / s;
    }
  } else {
    for (int n = 0; n <= nmax; ++n) F[n] = NAN;
  }
}

/* All derivatives d^m G(x), m in M(pmax), in nu order (D has N(pmax)). */
int or_derivatives(int kernel, int d, double lam, int pmax, const double* x,
                   double* D) {
  ld r2 = LDC(0.0), xl[OR_MAXD];
  for (int k = 0; k < d; ++k) {
    xl[k] = x[k];
    r2 += xl[k] * xl[k];
  }
  if (r2 == LDC(0.0)) return OR_ERR_DOMAIN;
  ld r = LD_SQRT(r2);
  ld* F = (ld*)malloc(sizeof(ld) * (pmax + 1));
  or_radial(kernel, d, lam, r, pmax, F);
  /* per-coordinate powers and the 1D Hermite weights */
  ld xp[OR_MAXD][80];
  for (int k = 0; k < d; ++k) {
    xp[k][0] = LDC(1.0);
    for (int e = 1; e <= pmax; ++e) xp[k][e] = xp[k][e - 1] * xl[k];
  }
  int nfull = or_num_terms(d, pmax);
  int* mi = (int*)malloc(sizeof(int) * nfull * d);
  or_multi_indices(d, pmax, mi);
  for (int l = 0; l < nfull; ++l) {
    const int* k = mi + l * d;
    int ktot = 0;
    for (int i = 0; i < d; ++i) ktot += k[i];
    /* iterate mu over the box 0 <= mu_i <= k_i/2 */
    int mu[OR_MAXD] = {0, 0, 0};
    ld sum = LDC(0.0);
    for (;;) {
      ld term = LDC(1.0);
      int mutot = 0;
      for (int i = 0; i < d; ++i) {
        /* k_i! / (mu_i! (k_i - 2 mu_i)! 2^mu_i) */
        ld c = LDC(1.0);
        for (int t = k[i] - 2 * mu[i] + 1; t <= k[i]; ++t) c *= (ld)t;
        for (int t = 2; t <= mu[i]; ++t) c /= (ld)t;
        for (int t = 0; t < mu[i]; ++t) c *= LDC(0.5);
        term *= c * xp[i][k[i] - 2 * mu[i]];
        mutot += mu[i];
      }
      sum += term * F[ktot - mutot];
      int i = 0;
      while (i < d) {
        if (2 * (mu[i] + 1) <= k[i]) {
          ++mu[i];
          break;
        }
        mu[i] = 0;
        ++i;
      }
      if (i == d) break;
    }
    D[l] = (double)sum;
  }
  free(mi);
  free(F);
  return OR_OK;
}

/* G(x) itself and its gradient (d_k G = x_k F'(s)), in plain double, for the
 * direct sums of eq. (1); reading R5 fixes the normalisations. */
static double or_green(int kernel, int d, double lam, const double* x) {
  double r2 = 0.0;
  for (int k = 0; k < d; ++k) r2 += x[k] * x[k];
  double r = sqrt(r2);
  if (kernel == OR_LAPLACE) return d == 3 ? 1.0 / (4.0 * M_PI * r) : log(r);
  if (kernel == OR_YUKAWA) return exp(-lam * r) / r;
  if (kernel == OR_HELM_RE) return cos(lam * r) / r;
  if (kernel == OR_HELM_IM) return sin(lam * r) / r;
  if (kernel == OR_BIHARMONIC) return d == 3 ? r : r2 * log(r);
  return NAN;
}

static void or_green_grad(int kernel, int d, double lam, const double* x,
                          double* g) {
  double r2 = 0.0;
  for (int k = 0; k < d; ++k) r2 += x[k] * x[k];
  double r = sqrt(r2), f1 = NAN; /* F'(s) = (1/r) dG/dr */
  if (kernel == OR_LAPLACE) f1 = d == 3 ? -1.0 / (4.0 * M_PI * r * r2) : 1.0 / r2;
  if (kernel == OR_YUKAWA) f1 = exp(-lam * r) * (-lam / r2 - 1.0 / (r * r2));
  if (kernel == OR_HELM_RE) f1 = -lam * sin(lam * r) / r2 - cos(lam * r) / (r * r2);
  if (kernel == OR_HELM_IM) f1 = lam * cos(lam * r) / r2 - sin(lam * r) / (r * r2);
  if (kernel == OR_BIHARMONIC) f1 = d == 3 ? 1.0 / r : 2.0 * log(r) + 1.0;
  for (int k = 0; k < d; ++k) g[k] = x[k] * f1;
}

/* ------------------------------------------------------------------------ */
/* Direct summation, eq. (1): phi(x) = sum_{y != x} G(x - y) w(y).           */
/* ------------------------------------------------------------------------ */

void or_direct(int kernel, int d, double lam, int64_t nsrc, const double* src,
               const double* w, int64_t ntgt, const double* tgt, double* phi,
               double* grad /* ntgt*d or NULL */) {
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t i = 0; i < ntgt; ++i) {
    double acc = 0.0, ga[OR_MAXD] = {0, 0, 0}, r[OR_MAXD], g[OR_MAXD];
    for (int64_t s = 0; s < nsrc; ++s) {
      int same = 1;
      for (int k = 0; k < d; ++k) {
        r[k] = tgt[i * d + k] - src[s * d + k];
        same &= (r[k] == 0.0);
      }
      if (same) continue; /* reading R6 */
      acc += or_green(kernel, d, lam, r) * w[s];
      if (grad) {
        or_green_grad(kernel, d, lam, r, g);
        for (int k = 0; k < d; ++k) ga[k] += g[k] * w[s];
      }
    }
    phi[i] = acc;
    if (grad)
      for (int k = 0; k < d; ++k) grad[i * d + k] = ga[k];
  }
}

/* ------------------------------------------------------------------------ */
/* Expansion operators (Secs. 2, 3.2-3.5, 4.1-4.3).                          */
/* ------------------------------------------------------------------------ */

/* P2M, Sec. 3.4: alpha_q = sum_y w (c - y)^q / q!, beta = M^T alpha. */
void or_p2m(const or_expansion* e, const double* c, int64_t n, const double* y,
            const double* w, double* beta) {
  int d = e->d, p = e->p;
  double* alpha = (double*)calloc(e->nfull, sizeof(double));
  double* qfact = (double*)malloc(sizeof(double) * e->nfull);
  for (int l = 0; l < e->nfull; ++l) qfact[l] = or_mi_factorial(d, e->mi + l * d);
  double pw[OR_MAXD][64];
  for (int64_t s = 0; s < n; ++s) {
    for (int k = 0; k < d; ++k) {
      pw[k][0] = 1.0;
      double u = c[k] - y[s * d + k];
      for (int t = 1; t <= p; ++t) pw[k][t] = pw[k][t - 1] * u;
    }
    for (int l = 0; l < e->nfull; ++l) {
      const int* q = e->mi + l * d;
      double v = w[s];
      for (int k = 0; k < d; ++k) v *= pw[k][q[k]];
      alpha[l] += v / qfact[l];
    }
  }
  or_compress(e, alpha, beta);
  free(qfact);
  free(alpha);
}

/* M2P, eq. (multipole_eval_beta): phi(x) = sum_{q in j} d^q G(x - c) beta_q. */
double or_m2p(const or_expansion* e, int kernel, double lam, const double* c,
              const double* beta, const double* x) {
  int d = e->d;
  double r[OR_MAXD];
  for (int k = 0; k < d; ++k) r[k] = x[k] - c[k];
  double* D = (double*)malloc(sizeof(double) * e->nfull);
  or_derivatives(kernel, d, lam, e->p, r, D);
  double acc = 0.0;
  for (int t = 0; t < e->nj; ++t) acc += D[e->j[t]] * beta[t];
  free(D);
  return acc;
}

/* Uncompressed M2M, eq. (mpole_translated_full_coeffs):
 * rho_q = sum_{i <= q} h^(q-i)/(q-i)! a_i,  h = c2 - c1 (a has nfull). */
void or_m2m_full(const or_expansion* e, const double* h, const double* a,
                 double* rho) {
  int d = e->d;
  for (int l = 0; l < e->nfull; ++l) {
    const int* q = e->mi + l * d;
    double acc = 0.0;
    for (int i = 0; i < e->nfull; ++i) {
      const int* m = e->mi + i * d;
      int le = 1;
      for (int k = 0; k < d; ++k) le &= (m[k] <= q[k]);
      if (!le || a[i] == 0.0) continue;
      double v = a[i];
      for (int k = 0; k < d; ++k) {
        int e2 = q[k] - m[k];
        for (int t = 1; t <= e2; ++t) v *= h[k] / (double)t;
      }
      acc += v;
    }
    rho[l] = acc;
  }
}

/* Compressed M2M, eqs. (mpole_translated_compressed_coeffs), (define_psi):
 * psi = M^T T E beta. */
void or_m2m(const or_expansion* e, const double* h, const double* beta,
            double* psi) {
  double* Eb = (double*)calloc(e->nfull, sizeof(double));
  double* sigma = (double*)malloc(sizeof(double) * e->nfull);
  for (int t = 0; t < e->nj; ++t) Eb[e->j[t]] = beta[t];
  or_m2m_full(e, h, Eb, sigma);
  or_compress(e, sigma, psi);
  free(Eb);
  free(sigma);
}

/* Compressed M2L, eq. (m2l_toeplitz) with reading R4 (no 1/nu(i)!):
 * L_i = sum_{q in j} d^{nu(i)+nu(q)} G(c2 - c1) beta_q  for i in j.
 * D2 holds d^m G(c2 - c1) for m in M(2p) in nu order. */
void or_m2l(const or_expansion* e, const double* D2, const double* beta,
            double* L) {
  int d = e->d, m[OR_MAXD];
  for (int a = 0; a < e->nj; ++a) {
    const int* ia = e->mi + e->j[a] * d;
    double acc = 0.0;
    for (int b = 0; b < e->nj; ++b) {
      const int* qb = e->mi + e->j[b] * d;
      for (int k = 0; k < d; ++k) m[k] = ia[k] + qb[k];
      acc += D2[or_mi_index(d, m)] * beta[b];
    }
    L[a] += acc;
  }
}

/* Uncompressed M2L (Sec. 2): L_r = sum_{|q|<=p} d^{r+q} G(c2 - c1) alpha_q
 * for every r in M(p) -- the naive O(p^{2d}) operator. */
void or_m2l_naive(int d, int p, const double* D2, const double* alpha,
                  double* L) {
  int nfull = or_num_terms(d, p);
  int* mi = (int*)malloc(sizeof(int) * nfull * d);
  or_multi_indices(d, p, mi);
  int m[OR_MAXD];
  for (int a = 0; a < nfull; ++a) {
    double acc = 0.0;
    for (int b = 0; b < nfull; ++b) {
      for (int k = 0; k < d; ++k) m[k] = mi[a * d + k] + mi[b * d + k];
      acc += D2[or_mi_index(d, m)] * alpha[b];
    }
    L[a] = acc;
  }
  free(mi);
}

/* Compressed L2L, eq. (l2l-expr) with reading R4: with D = M L1 the full
 * derivative vector at c1 and h = c2 - c1,
 * L2_i = sum_{q >= i} D_q h^(q-i)/(q-i)!   for i in j. */
void or_l2l(const or_expansion* e, const double* h, const double* L1,
            double* L2) {
  int d = e->d;
  double* D = (double*)malloc(sizeof(double) * e->nfull);
  or_decompress(e, L1, D);
  for (int a = 0; a < e->nj; ++a) {
    const int* i = e->mi + e->j[a] * d;
    double acc = 0.0;
    for (int l = 0; l < e->nfull; ++l) {
      const int* q = e->mi + l * d;
      int ge = 1;
      for (int k = 0; k < d; ++k) ge &= (q[k] >= i[k]);
      if (!ge) continue;
      double v = D[l];
      for (int k = 0; k < d; ++k) {
        int e2 = q[k] - i[k];
        for (int t = 1; t <= e2; ++t) v *= h[k] / (double)t;
      }
      acc += v;
    }
    L2[a] += acc;
  }
  free(D);
}

/* L2P, Sec. 3.3: phi(x) = sum_m [M L]_m / m! (x - c)^m; optional gradient. */
double or_l2p(const or_expansion* e, const double* c, const double* L,
              const double* x, double* grad) {
  int d = e->d, p = e->p;
  double* D = (double*)malloc(sizeof(double) * e->nfull);
  or_decompress(e, L, D);
  double u[OR_MAXD], pw[OR_MAXD][64];
  for (int k = 0; k < d; ++k) {
    u[k] = x[k] - c[k];
    pw[k][0] = 1.0;
    for (int t = 1; t <= p; ++t) pw[k][t] = pw[k][t - 1] * u[k];
  }
  double phi = 0.0, g[OR_MAXD] = {0, 0, 0};
  for (int l = 0; l < e->nfull; ++l) {
    const int* m = e->mi + l * d;
    double a = D[l] / or_mi_factorial(d, m);
    double v = a;
    for (int k = 0; k < d; ++k) v *= pw[k][m[k]];
    phi += v;
    if (grad) {
      for (int k = 0; k < d; ++k) {
        if (m[k] == 0) continue;
        double gv = a * (double)m[k];
        for (int k2 = 0; k2 < d; ++k2) gv *= pw[k2][m[k2] - (k2 == k ? 1 : 0)];
        g[k] += gv;
      }
    }
  }
  if (grad)
    for (int k = 0; k < d; ++k) grad[k] = g[k];
  free(D);
  return phi;
}

/* P2L, eq. (stored_local_coeffs): L_i = sum_y d^{nu(i)} G(c - y) w, i in j. */
void or_p2l(const or_expansion* e, int kernel, double lam, const double* c,
            int64_t n, const double* y, const double* w, double* L) {
  int d = e->d;
  double* D = (double*)malloc(sizeof(double) * e->nfull);
  double r[OR_MAXD];
  for (int64_t s = 0; s < n; ++s) {
    for (int k = 0; k < d; ++k) r[k] = c[k] - y[s * d + k];
    or_derivatives(kernel, d, lam, e->p, r, D);
    for (int t = 0; t < e->nj; ++t) L[t] += D[e->j[t]] * w[s];
  }
  free(D);
}

/* ------------------------------------------------------------------------ */
/* Uniform-tree FMM driver (Sec. 1 and reading R7).  Boxes at level l are    */
/* numbered lexicographically, x fastest; box b has centre                   */
/* lo + (b + 1/2) size/2^l.                                                   */
/* ------------------------------------------------------------------------ */

typedef struct {
  int kernel, d, p, L, c, compressed;
  double lam, lo[OR_MAXD], size;
} or_fmm_cfg;

static int64_t or_nbox(int d, int l) { return (int64_t)1 << (d * l); }

static void or_box_coords(int d, int l, int64_t b, int* bc) {
  int64_t n = (int64_t)1 << l;
  for (int k = 0; k < d; ++k) {
    bc[k] = (int)(b % n);
    b /= n;
  }
}

static int64_t or_box_index(int d, int l, const int* bc) {
  int64_t n = (int64_t)1 << l, b = 0;
  for (int k = d - 1; k >= 0; --k) b = b * n + bc[k];
  return b;
}

static void or_box_center(const or_fmm_cfg* f, int l, const int* bc, double* c) {
  double s = f->size / (double)((int64_t)1 << l);
  for (int k = 0; k < f->d; ++k) c[k] = f->lo[k] + (bc[k] + 0.5) * s;
}

/* Leaf box of every point; returns OR_ERR_DOMAIN if a point is outside. */
static int or_bin(const or_fmm_cfg* f, int64_t n, const double* x, int64_t* box) {
  int64_t nl = (int64_t)1 << f->L;
  double s = f->size / (double)nl;
  for (int64_t i = 0; i < n; ++i) {
    int bc[OR_MAXD];
    for (int k = 0; k < f->d; ++k) {
      double t = (x[i * f->d + k] - f->lo[k]) / s;
      if (!(t >= 0.0) || t > (double)nl) return OR_ERR_DOMAIN;
      int64_t b = (int64_t)floor(t);
      if (b >= nl) b = nl - 1;
      bc[k] = (int)b;
    }
    box[i] = or_box_index(f->d, f->L, bc);
  }
  return OR_OK;
}

/* Bucket point indices by box: start[nb+1], idx[n] (stable). */
static void or_bucket(int64_t nb, int64_t n, const int64_t* box, int64_t* start,
                      int64_t* idx) {
  for (int64_t b = 0; b <= nb; ++b) start[b] = 0;
  for (int64_t i = 0; i < n; ++i) start[box[i] + 1]++;
  for (int64_t b = 0; b < nb; ++b) start[b + 1] += start[b];
  int64_t* cur = (int64_t*)malloc(sizeof(int64_t) * nb);
  for (int64_t b = 0; b < nb; ++b) cur[b] = start[b];
  for (int64_t i = 0; i < n; ++i) idx[cur[box[i]]++] = i;
  free(cur);
}

/* Full uniform FMM.  If nsample > 0, only the targets listed in sample[] are
 * evaluated (phi/grad then have nsample entries, in sample order); the
 * multipoles are still formed for every box.  Returns OR_OK or an error. */
int or_fmm_uniform(int kernel, int d, double lam, int p, int L, int compressed,
                   const double* lo, double size, int64_t nsrc, const double* src,
                   const double* w, int64_t ntgt, const double* tgt,
                   int64_t nsample, const int64_t* sample, double* phi,
                   double* grad) {
  if (d < 2 || d > 3 || p < 0 || L < 2 || size <= 0.0) return OR_ERR_ARG;
  or_fmm_cfg f;
  f.kernel = kernel;
  f.d = d;
  f.p = p;
  f.L = L;
  f.lam = lam;
  f.size = size;
  f.compressed = compressed;
  for (int k = 0; k < d; ++k) f.lo[k] = lo[k];
  double acoef[64];
  f.c = or_pde_for_kernel(kernel, d, lam, acoef);
  if (f.c < 0) return OR_ERR_UNSUPPORTED;
  or_expansion* e = or_expansion_new(d, p, f.c, acoef, compressed);
  int nj = e->nj;

  int64_t nleaf = or_nbox(d, L);
  int64_t* sbox = (int64_t*)malloc(sizeof(int64_t) * (nsrc > 0 ? nsrc : 1));
  int64_t* tbox = (int64_t*)malloc(sizeof(int64_t) * (ntgt > 0 ? ntgt : 1));
  if (or_bin(&f, nsrc, src, sbox) != OR_OK || or_bin(&f, ntgt, tgt, tbox) != OR_OK) {
    free(sbox);
    free(tbox);
    or_expansion_free(e);
    return OR_ERR_DOMAIN;
  }
  int64_t* sstart = (int64_t*)malloc(sizeof(int64_t) * (nleaf + 1));
  int64_t* sidx = (int64_t*)malloc(sizeof(int64_t) * (nsrc > 0 ? nsrc : 1));
  or_bucket(nleaf, nsrc, sbox, sstart, sidx);

  /* expansions per level */
  double* mp[32];
  double* lc[32];
  char* need[32];
  for (int l = 0; l <= L; ++l) {
    mp[l] = (double*)calloc((size_t)or_nbox(d, l) * nj, sizeof(double));
    lc[l] = (double*)calloc((size_t)or_nbox(d, l) * nj, sizeof(double));
    need[l] = (char*)calloc((size_t)or_nbox(d, l), 1);
  }
  /* which boxes need a local expansion: all, or the sampled targets' chain */
  int64_t neval = nsample > 0 ? nsample : ntgt;
  for (int64_t t = 0; t < neval; ++t) {
    int64_t it = nsample > 0 ? sample[t] : t;
    int bc[OR_MAXD];
    or_box_coords(d, L, tbox[it], bc);
    for (int l = L; l >= 0; --l) {
      need[l][or_box_index(d, l, bc)] = 1;
      for (int k = 0; k < d; ++k) bc[k] >>= 1;
    }
  }

  /* P2M at the leaves (Sec. 3.4) */
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t b = 0; b < nleaf; ++b) {
    int64_t n = sstart[b + 1] - sstart[b];
    if (n == 0) continue;
    double* ys = (double*)malloc(sizeof(double) * n * d);
    double* ws = (double*)malloc(sizeof(double) * n);
    for (int64_t s = 0; s < n; ++s) {
      int64_t i = sidx[sstart[b] + s];
      for (int k = 0; k < d; ++k) ys[s * d + k] = src[i * d + k];
      ws[s] = w[i];
    }
    int bc[OR_MAXD];
    double c[OR_MAXD];
    or_box_coords(d, L, b, bc);
    or_box_center(&f, L, bc, c);
    or_p2m(e, c, n, ys, ws, mp[L] + (size_t)b * nj);
    free(ys);
    free(ws);
  }

  /* M2M, levels L-1 .. 2 (Sec. 4.3): psi = M^T T E beta per child */
  for (int l = L - 1; l >= 2; --l) {
    int64_t nb = or_nbox(d, l);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t b = 0; b < nb; ++b) {
      int bc[OR_MAXD], cc[OR_MAXD];
      double cp[OR_MAXD], ch[OR_MAXD], h[OR_MAXD];
      double* psi = (double*)malloc(sizeof(double) * nj);
      or_box_coords(d, l, b, bc);
      or_box_center(&f, l, bc, cp);
      for (int ci = 0; ci < (1 << d); ++ci) {
        for (int k = 0; k < d; ++k) cc[k] = 2 * bc[k] + ((ci >> k) & 1);
        int64_t cb = or_box_index(d, l + 1, cc);
        or_box_center(&f, l + 1, cc, ch);
        for (int k = 0; k < d; ++k) h[k] = cp[k] - ch[k];
        or_m2m(e, h, mp[l + 1] + (size_t)cb * nj, psi);
        for (int t = 0; t < nj; ++t) mp[l][(size_t)b * nj + t] += psi[t];
      }
      free(psi);
    }
  }

  /* M2L, levels 2..L (Sec. 4.1).  The derivatives depend only on c2 - c1,
   * so they are formed once per level for every offset in [-3,3]^d. */
  int noff1 = 7, noff = 1;
  for (int k = 0; k < d; ++k) noff *= noff1;
  int n2 = or_num_terms(d, 2 * p);
  double* D2 = (double*)malloc(sizeof(double) * (size_t)noff * n2);
  for (int l = 2; l <= L; ++l) {
    double s = f.size / (double)((int64_t)1 << l);
#pragma omp parallel for schedule(dynamic, 1)
    for (int o = 0; o < noff; ++o) {
      int oc[OR_MAXD], t = o, far = 0;
      double hv[OR_MAXD];
      for (int k = 0; k < d; ++k) {
        oc[k] = t % noff1 - 3;
        t /= noff1;
        if (oc[k] > 1 || oc[k] < -1) far = 1;
        hv[k] = oc[k] * s;
      }
      if (far) or_derivatives(kernel, d, lam, 2 * p, hv, D2 + (size_t)o * n2);
    }
    int64_t nb = or_nbox(d, l);
    int64_t n = (int64_t)1 << l;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t b = 0; b < nb; ++b) {
      if (!need[l][b]) continue;
      int bc[OR_MAXD], pc[OR_MAXD];
      or_box_coords(d, l, b, bc);
      for (int k = 0; k < d; ++k) pc[k] = bc[k] >> 1;
      /* children of the parent's neighbours (parent included) */
      int nn = 1;
      for (int k = 0; k < d; ++k) nn *= 6;
      for (int a = 0; a < nn; ++a) {
        int sc[OR_MAXD], tt = a, adj = 1, ok = 1;
        for (int k = 0; k < d; ++k) {
          sc[k] = 2 * (pc[k] - 1) + tt % 6;
          tt /= 6;
          if (sc[k] < 0 || sc[k] >= n) ok = 0;
          int dd = bc[k] - sc[k];
          if (dd > 1 || dd < -1) adj = 0;
        }
        if (!ok || adj) continue;
        int o = 0;
        for (int k = d - 1; k >= 0; --k) o = o * noff1 + (bc[k] - sc[k] + 3);
        int64_t sb = or_box_index(d, l, sc);
        or_m2l(e, D2 + (size_t)o * n2, mp[l] + (size_t)sb * nj,
               lc[l] + (size_t)b * nj);
      }
    }
  }
  free(D2);

  /* L2L, levels 2 .. L-1 -> children (Sec. 4.2) */
  for (int l = 2; l < L; ++l) {
    int64_t nb = or_nbox(d, l + 1);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t b = 0; b < nb; ++b) {
      if (!need[l + 1][b]) continue;
      int cc[OR_MAXD], pc[OR_MAXD];
      double cch[OR_MAXD], cpa[OR_MAXD], h[OR_MAXD];
      or_box_coords(d, l + 1, b, cc);
      for (int k = 0; k < d; ++k) pc[k] = cc[k] >> 1;
      or_box_center(&f, l + 1, cc, cch);
      or_box_center(&f, l, pc, cpa);
      for (int k = 0; k < d; ++k) h[k] = cch[k] - cpa[k];
      or_l2l(e, h, lc[l] + (size_t)or_box_index(d, l, pc) * nj,
             lc[l + 1] + (size_t)b * nj);
    }
  }

  /* L2P + P2P at the leaves */
  int64_t nl1 = (int64_t)1 << L;
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t t = 0; t < neval; ++t) {
    int64_t it = nsample > 0 ? sample[t] : t;
    const double* x = tgt + it * d;
    int bc[OR_MAXD];
    double c[OR_MAXD], g[OR_MAXD] = {0, 0, 0};
    or_box_coords(d, L, tbox[it], bc);
    or_box_center(&f, L, bc, c);
    double acc = or_l2p(e, c, lc[L] + (size_t)tbox[it] * nj, x, grad ? g : NULL);
    /* near field: the 3^d adjacent leaves, the box itself included */
    int nn = 1;
    for (int k = 0; k < d; ++k) nn *= 3;
    for (int a = 0; a < nn; ++a) {
      int sc[OR_MAXD], tt = a, ok = 1;
      for (int k = 0; k < d; ++k) {
        sc[k] = bc[k] - 1 + tt % 3;
        tt /= 3;
        if (sc[k] < 0 || sc[k] >= nl1) ok = 0;
      }
      if (!ok) continue;
      int64_t sb = or_box_index(d, L, sc);
      for (int64_t q = sstart[sb]; q < sstart[sb + 1]; ++q) {
        int64_t is = sidx[q];
        double r[OR_MAXD], gg[OR_MAXD];
        int same = 1;
        for (int k = 0; k < d; ++k) {
          r[k] = x[k] - src[is * d + k];
          same &= (r[k] == 0.0);
        }
        if (same) continue;
        acc += or_green(kernel, d, lam, r) * w[is];
        if (grad) {
          or_green_grad(kernel, d, lam, r, gg);
          for (int k = 0; k < d; ++k) g[k] += gg[k] * w[is];
        }
      }
    }
    phi[t] = acc;
    if (grad)
      for (int k = 0; k < d; ++k) grad[t * d + k] = g[k];
  }

  for (int l = 0; l <= L; ++l) {
    free(mp[l]);
    free(lc[l]);
    free(need[l]);
  }
  free(sbox);
  free(tbox);
  free(sstart);
  free(sidx);
  or_expansion_free(e);
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Adaptive-tree FMM (reading R15).  The tree refines a box of the root cube  */
/* while it holds more than max_leaf points (sources plus targets) and its    */
/* level is below max_depth; children that would hold no point are not       */
/* created.  "Adjacent" means the closed boxes touch or coincide.  For a box  */
/* B of level l with parent P(B), the interaction lists are, by definition    */
/* (the classical adaptive FMM; the paper's List 2 is V):                     */
/*   U(B), B a leaf: the leaves adjacent to B, B included         -> P2P      */
/*   V(B), l >= 2:   boxes C of level l with P(C) adjacent to P(B) and C not  */
/*                   adjacent to B                                -> M2L      */
/*   W(B), B a leaf: boxes C with level(C) > l, P(C) adjacent to B and C not  */
/*                   adjacent to B                                -> M2P      */
/*   X(B), l >= 2:   leaves A with level(A) < l, A adjacent to P(B) and A not */
/*                   adjacent to B (exactly the A with B in W(A)) -> P2L      */
/* Local expansions live at levels >= 2: L2L from the parent, plus M2L over V */
/* and P2L over X.  Every leaf evaluates L2P, P2P over U and M2P over W.      */
/* A W or X interaction is summed directly (P2P) when the box on the far side */
/* holds no more points than an expansion has coefficients (|j|): a W box C  */
/* with at most |j| sources is summed at the leaf's targets in place of M2P;  */
/* an X pair (A, B) whose box B holds at most |j| targets (its whole subtree) */
/* sends A's sources straight to those targets in place of P2L.  The choice   */
/* depends on one box's count only, so every target gets each pair once.     */
/* The lists are found by testing their definitions against every box.       */
/* ------------------------------------------------------------------------ */

typedef struct {
  int level, leaf;
  int64_t c[OR_MAXD];
  int64_t parent;
  int64_t child0, nchild; /* children: boxes child0 .. child0+nchild-1, Morton order */
  int64_t s0, s1, t0, t1; /* ranges in the Morton-sorted source / target orders */
} or_abox;

static int or_abox_adjacent(int d, const or_abox* A, const or_abox* B) {
  int m = A->level > B->level ? A->level : B->level;
  for (int k = 0; k < d; ++k) {
    int64_t a0 = A->c[k] << (m - A->level), a1 = (A->c[k] + 1) << (m - A->level);
    int64_t b0 = B->c[k] << (m - B->level), b1 = (B->c[k] + 1) << (m - B->level);
    if (a0 > b1 || b0 > a1) return 0;
  }
  return 1;
}

static void or_abox_center(int d, const double* lo, double size, const or_abox* B, double* c) {
  double s = size / (double)((int64_t)1 << B->level);
  for (int k = 0; k < d; ++k) c[k] = lo[k] + (B->c[k] + 0.5) * s;
}

/* Morton key of a point at depth D (per level, the bit of axis k at position k). */
static int or_morton(int d, int D, const double* lo, double size, const double* x,
                     uint64_t* key) {
  int64_t n = (int64_t)1 << D;
  double s = size / (double)n;
  int64_t kc[OR_MAXD];
  for (int k = 0; k < d; ++k) {
    double t = (x[k] - lo[k]) / s;
    if (!(t >= 0.0) || t > (double)n) return OR_ERR_DOMAIN;
    int64_t b = (int64_t)floor(t);
    if (b >= n) b = n - 1;
    kc[k] = b;
  }
  uint64_t m = 0;
  for (int b = D - 1; b >= 0; --b) {
    uint64_t dig = 0;
    for (int k = 0; k < d; ++k) dig |= (uint64_t)((kc[k] >> b) & 1) << k;
    m = (m << d) | dig;
  }
  *key = m;
  return OR_OK;
}

typedef struct {
  uint64_t key;
  int64_t idx;
} or_keyed;

static int or_keyed_cmp(const void* a, const void* b) {
  const or_keyed* x = (const or_keyed*)a;
  const or_keyed* y = (const or_keyed*)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  return x->idx < y->idx ? -1 : (x->idx > y->idx);
}

static int or_sort_points(int d, int D, const double* lo, double size, int64_t n,
                          const double* x, or_keyed* out) {
  for (int64_t i = 0; i < n; ++i) {
    out[i].idx = i;
    if (or_morton(d, D, lo, size, x + i * d, &out[i].key) != OR_OK) return OR_ERR_DOMAIN;
  }
  qsort(out, (size_t)n, sizeof(or_keyed), or_keyed_cmp);
  return OR_OK;
}

/* Adaptive FMM (3D and 2D).  If nsample > 0 only the listed targets are
 * evaluated (outputs in sample order).  stats (optional, 8 entries): boxes,
 * leaves, deepest level, then |U|, |V|, |W|, |X| summed over the boxes that
 * the evaluated targets use, and how many of the W and X pairs among them were
 * summed directly.  cover (optional, one per evaluated target):
 * the number of sources the lists of that target's leaf and ancestors reach,
 * with multiplicity (exactly n_src when every pair is covered once and no
 * source coincides with the target). */
int or_fmm_adaptive(int kernel, int d, double lam, int p, int max_leaf, int max_depth,
                    const double* lo, double size, int64_t nsrc, const double* src,
                    const double* w, int64_t ntgt, const double* tgt, int64_t nsample,
                    const int64_t* sample, double* phi, int64_t* stats, double* cover) {
  if (d < 2 || d > 3 || p < 0 || max_leaf < 1 || max_depth < 0 || max_depth > 20 ||
      size <= 0.0)
    return OR_ERR_ARG;
  double acoef[64];
  int c = or_pde_for_kernel(kernel, d, lam, acoef);
  if (c < 0) return OR_ERR_UNSUPPORTED;
  const int D = max_depth, nch = 1 << d;
  or_keyed* ss = (or_keyed*)malloc(sizeof(or_keyed) * (nsrc > 0 ? nsrc : 1));
  or_keyed* ts = (or_keyed*)malloc(sizeof(or_keyed) * (ntgt > 0 ? ntgt : 1));
  if (or_sort_points(d, D, lo, size, nsrc, src, ss) != OR_OK ||
      or_sort_points(d, D, lo, size, ntgt, tgt, ts) != OR_OK) {
    free(ss);
    free(ts);
    return OR_ERR_DOMAIN;
  }

  /* tree, breadth first (children appended in Morton order) */
  int64_t cap = 1024, nbox = 1;
  or_abox* bx = (or_abox*)malloc(sizeof(or_abox) * cap);
  memset(&bx[0], 0, sizeof(or_abox));
  bx[0].parent = -1;
  bx[0].s1 = nsrc;
  bx[0].t1 = ntgt;
  int maxlev = 0;
  for (int64_t b = 0; b < nbox; ++b) {
    int64_t npt = (bx[b].s1 - bx[b].s0) + (bx[b].t1 - bx[b].t0);
    if (npt <= max_leaf || bx[b].level >= D) {
      bx[b].leaf = 1;
      continue;
    }
    const int shift = d * (D - bx[b].level - 1);
    int64_t si = bx[b].s0, ti = bx[b].t0;
    bx[b].child0 = nbox;
    for (int ci = 0; ci < nch; ++ci) {
      int64_t s0 = si, t0 = ti;
      while (si < bx[b].s1 && (int)((ss[si].key >> shift) & (uint64_t)(nch - 1)) == ci) ++si;
      while (ti < bx[b].t1 && (int)((ts[ti].key >> shift) & (uint64_t)(nch - 1)) == ci) ++ti;
      if (si == s0 && ti == t0) continue;
      if (nbox == cap) {
        cap *= 2;
        bx = (or_abox*)realloc(bx, sizeof(or_abox) * cap);
      }
      or_abox* ch = &bx[nbox++];
      memset(ch, 0, sizeof(or_abox));
      ch->level = bx[b].level + 1;
      for (int k = 0; k < d; ++k) ch->c[k] = 2 * bx[b].c[k] + ((ci >> k) & 1);
      ch->parent = b;
      ch->s0 = s0;
      ch->s1 = si;
      ch->t0 = t0;
      ch->t1 = ti;
      if (ch->level > maxlev) maxlev = ch->level;
    }
    bx[b].nchild = nbox - bx[b].child0;
  }
  /* leaf of every sorted target position */
  int64_t* tleaf = (int64_t*)malloc(sizeof(int64_t) * (ntgt > 0 ? ntgt : 1));
  int64_t* tpos = (int64_t*)malloc(sizeof(int64_t) * (ntgt > 0 ? ntgt : 1));
  for (int64_t b = 0; b < nbox; ++b)
    if (bx[b].leaf)
      for (int64_t t = bx[b].t0; t < bx[b].t1; ++t) tleaf[t] = b;
  for (int64_t t = 0; t < ntgt; ++t) tpos[ts[t].idx] = t;

  or_expansion* e = or_expansion_new(d, p, c, acoef, 1);
  const int nj = e->nj;
  const size_t nbx = (size_t)(nbox > 0 ? nbox : 1);
  double* mp = (double*)calloc(nbx * nj, sizeof(double));
  double* lc = (double*)calloc(nbx * nj, sizeof(double));
  char* need = (char*)calloc(nbx, 1);
  double* vxcov = (double*)calloc(nbx, sizeof(double));
  int64_t cnt[5] = {0, 0, 0, 0, 0};

  const int64_t neval = nsample > 0 ? nsample : ntgt;
  for (int64_t t = 0; t < neval; ++t) {
    int64_t it = nsample > 0 ? sample[t] : t;
    for (int64_t b = tleaf[tpos[it]]; b >= 0; b = bx[b].parent) need[b] = 1;
  }

  /* P2M at the leaves of level >= 2 (Sec. 3.4) */
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t b = 0; b < nbox; ++b) {
    if (!bx[b].leaf || bx[b].level < 2 || bx[b].s1 == bx[b].s0) continue;
    int64_t n = bx[b].s1 - bx[b].s0;
    double* ys = (double*)malloc(sizeof(double) * n * d);
    double* ws = (double*)malloc(sizeof(double) * n);
    for (int64_t q = 0; q < n; ++q) {
      int64_t i = ss[bx[b].s0 + q].idx;
      for (int k = 0; k < d; ++k) ys[q * d + k] = src[i * d + k];
      ws[q] = w[i];
    }
    double cb[OR_MAXD];
    or_abox_center(d, lo, size, &bx[b], cb);
    or_p2m(e, cb, n, ys, ws, mp + (size_t)b * nj);
    free(ys);
    free(ws);
  }
  /* M2M, deepest level first (Sec. 4.3): every parent of level l-1 adds the
   * translated multipoles of its children in Morton order, so the sum runs in
   * the same order whatever the number of threads */
  for (int l = maxlev; l >= 3; --l) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t pb = 0; pb < nbox; ++pb) {
      if (bx[pb].level != l - 1 || bx[pb].leaf) continue;
      double cp[OR_MAXD], cb[OR_MAXD], h[OR_MAXD];
      or_abox_center(d, lo, size, &bx[pb], cp);
      double* psi = (double*)malloc(sizeof(double) * nj);
      for (int64_t b = bx[pb].child0; b < bx[pb].child0 + bx[pb].nchild; ++b) {
        or_abox_center(d, lo, size, &bx[b], cb);
        for (int k = 0; k < d; ++k) h[k] = cp[k] - cb[k];
        or_m2m(e, h, mp + (size_t)b * nj, psi);
        for (int t = 0; t < nj; ++t) mp[(size_t)pb * nj + t] += psi[t];
      }
      free(psi);
    }
  }

  /* M2L derivative tables per level and offset in [-3,3]^d (Sec. 4.1) */
  int noff = 1;
  for (int k = 0; k < d; ++k) noff *= 7;
  const int n2 = or_num_terms(d, 2 * p);
  double* D2 = (double*)calloc((size_t)(maxlev + 1) * noff * n2, sizeof(double));
  for (int l = 2; l <= maxlev; ++l) {
    double s = size / (double)((int64_t)1 << l);
#pragma omp parallel for schedule(dynamic, 1)
    for (int o = 0; o < noff; ++o) {
      int t = o, far = 0;
      double hv[OR_MAXD];
      for (int k = 0; k < d; ++k) {
        int oc = t % 7 - 3;
        t /= 7;
        if (oc > 1 || oc < -1) far = 1;
        hv[k] = oc * s;
      }
      if (far) or_derivatives(kernel, d, lam, 2 * p, hv, D2 + ((size_t)l * noff + o) * n2);
    }
  }

  /* local expansions, coarse to fine: L2L + M2L over V + P2L over X */
  for (int l = 2; l <= maxlev; ++l) {
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t b = 0; b < nbox; ++b) {
      if (bx[b].level != l || !need[b]) continue;
      double cb[OR_MAXD];
      or_abox_center(d, lo, size, &bx[b], cb);
      double* Lb = lc + (size_t)b * nj;
      const int64_t pb = bx[b].parent;
      if (bx[pb].level >= 2) {
        double cp[OR_MAXD], h[OR_MAXD];
        or_abox_center(d, lo, size, &bx[pb], cp);
        for (int k = 0; k < d; ++k) h[k] = cb[k] - cp[k];
        or_l2l(e, h, lc + (size_t)pb * nj, Lb);
      }
      int64_t nv = 0, nx = 0, nxd = 0;
      double cov = 0.0;
      for (int64_t a = 0; a < nbox; ++a) {
        const or_abox* A = &bx[a];
        if (A->level == l && a != b && A->parent >= 0 &&
            or_abox_adjacent(d, &bx[A->parent], &bx[pb]) && !or_abox_adjacent(d, A, &bx[b])) {
          /* V: M2L (eq. (m2l_toeplitz)) */
          int o = 0;
          for (int k = d - 1; k >= 0; --k) o = o * 7 + (int)(bx[b].c[k] - A->c[k] + 3);
          or_m2l(e, D2 + ((size_t)l * noff + o) * n2, mp + (size_t)a * nj, Lb);
          cov += (double)(A->s1 - A->s0);
          ++nv;
        } else if (A->leaf && A->level < l && or_abox_adjacent(d, A, &bx[pb]) &&
                   !or_abox_adjacent(d, A, &bx[b])) {
          /* X: P2L (eq. (stored_local_coeffs)); with at most |j| targets
           * under B the leaves sum A's sources directly instead */
          int64_t n = A->s1 - A->s0;
          ++nx;
          if (bx[b].t1 - bx[b].t0 <= nj) {
            ++nxd;
            continue;
          }
          if (n > 0) {
            double* ys = (double*)malloc(sizeof(double) * n * d);
            double* ws = (double*)malloc(sizeof(double) * n);
            for (int64_t q = 0; q < n; ++q) {
              int64_t i = ss[A->s0 + q].idx;
              for (int k = 0; k < d; ++k) ys[q * d + k] = src[i * d + k];
              ws[q] = w[i];
            }
            or_p2l(e, kernel, lam, cb, n, ys, ws, Lb);
            free(ys);
            free(ws);
          }
          cov += (double)n;
        }
      }
      vxcov[b] = cov + vxcov[pb];
#pragma omp atomic
      cnt[1] += nv;
#pragma omp atomic
      cnt[3] += nx;
#pragma omp atomic
      cnt[4] += nxd;
    }
  }

  /* leaves: L2P + P2P over U + M2P over W */
  char* leafdone = (char*)calloc(nbx, 1);
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t t = 0; t < neval; ++t) {
    int64_t it = nsample > 0 ? sample[t] : t;
    const int64_t b = tleaf[tpos[it]];
    const or_abox* B = &bx[b];
    const double* x = tgt + it * d;
    double cb[OR_MAXD];
    or_abox_center(d, lo, size, B, cb);
    double acc = B->level >= 2 ? or_l2p(e, cb, lc + (size_t)b * nj, x, NULL) : 0.0;
    double cov = B->level >= 2 ? vxcov[b] : 0.0;
    int64_t nu = 0, nw = 0, nwd = 0;
    /* direct sum (eq. (1)) of the sources of box A at x, skipping x itself */
    #define OR_DIRECT(A)                                                     \
      for (int64_t q = (A)->s0; q < (A)->s1; ++q) {                          \
        int64_t is = ss[q].idx;                                              \
        double r[OR_MAXD];                                                   \
        int same = 1;                                                        \
        for (int k = 0; k < d; ++k) {                                        \
          r[k] = x[k] - src[is * d + k];                                     \
          same &= (r[k] == 0.0);                                             \
        }                                                                    \
        if (same) continue;                                                  \
        acc += or_green(kernel, d, lam, r) * w[is];                          \
        cov += 1.0;                                                          \
      }
    for (int64_t a = 0; a < nbox; ++a) {
      const or_abox* A = &bx[a];
      if (A->leaf && or_abox_adjacent(d, A, B)) {
        OR_DIRECT(A)
        ++nu;
      } else if (A->level > B->level && A->parent >= 0 &&
                 or_abox_adjacent(d, &bx[A->parent], B) && !or_abox_adjacent(d, A, B)) {
        if (A->s1 - A->s0 <= nj) {
          OR_DIRECT(A)  /* W box with at most |j| sources */
          ++nwd;
        } else {
          double ca[OR_MAXD];
          or_abox_center(d, lo, size, A, ca);
          acc += or_m2p(e, kernel, lam, ca, mp + (size_t)a * nj, x);
          cov += (double)(A->s1 - A->s0);
        }
        ++nw;
      }
    }
    /* X pairs (A, C) of the leaf's ancestors C (and the leaf) of level >= 2
     * holding at most |j| targets: A's sources directly */
    for (int64_t cbx = b; cbx >= 0 && bx[cbx].level >= 2 && bx[cbx].t1 - bx[cbx].t0 <= nj;
         cbx = bx[cbx].parent) {
      const or_abox* C = &bx[cbx];
      const or_abox* PC = &bx[C->parent];
      for (int64_t a = 0; a < nbox; ++a) {
        const or_abox* A = &bx[a];
        if (A->leaf && A->level < C->level && or_abox_adjacent(d, A, PC) &&
            !or_abox_adjacent(d, A, C)) {
          OR_DIRECT(A)
        }
      }
    }
    #undef OR_DIRECT
    phi[t] = acc;
    if (cover) cover[t] = cov;
    int first = 0;
#pragma omp critical
    {
      if (!leafdone[b]) {
        leafdone[b] = 1;
        first = 1;
      }
    }
    if (first) {
#pragma omp atomic
      cnt[0] += nu;
#pragma omp atomic
      cnt[2] += nw;
#pragma omp atomic
      cnt[4] += nwd;
    }
  }
  if (stats) {
    int64_t nleaf = 0;
    for (int64_t b = 0; b < nbox; ++b) nleaf += bx[b].leaf;
    stats[0] = nbox;
    stats[1] = nleaf;
    stats[2] = maxlev;
    stats[3] = cnt[0];
    stats[4] = cnt[1];
    stats[5] = cnt[2];
    stats[6] = cnt[3];
    stats[7] = cnt[4];
  }
  free(leafdone);
  free(D2);
  free(mp);
  free(lc);
  free(need);
  free(vxcov);
  free(tleaf);
  free(tpos);
  free(bx);
  free(ss);
  free(ts);
  or_expansion_free(e);
  return OR_OK;
}

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void or_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* Batched form of or_derivatives for n points (D is n x N(pmax)). */
int or_derivatives_batch(int kernel, int d, double lam, int pmax, int64_t n,
                         const double* x, double* D) {
  int nfull = or_num_terms(d, pmax), bad = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(| : bad)
  for (int64_t i = 0; i < n; ++i)
    bad |= (or_derivatives(kernel, d, lam, pmax, x + i * d, D + i * nfull) != OR_OK);
  return bad ? OR_ERR_DOMAIN : OR_OK;
}
