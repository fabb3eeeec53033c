/*
 * Independent CPU oracle for the power-series Newton step in multiple-double
 * arithmetic.  TEST INFRASTRUCTURE ONLY: it is used by tests/, by the smoke
 * check and by the benchmark's cpu_baseline / reference arm.  The product
 * path never links, loads or calls it, and this file shares no code, header
 * or table with the CUDA library.
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math -fopenmp -shared -fPIC.
 * Contraction is off so that every +,-,* is a separately rounded binary64
 * operation; fused multiply-adds appear only where fma() is written.
 * With -DORACLE_COUNT every binary64 operation is counted (op-count pins).
 *
 * What is computed, with its source in the paper (arXiv 2012.06607):
 *   Sec. 2, Table 1   multiple-double (md) numbers: unevaluated sums of K
 *                     doubles, K in {1,2,3,4,5,8,10}; add, mul, div.
 *   Sec. 2            md square root (needed by the 2-norm example of Sec. 2).
 *   Sec. 3            truncated series product: (d+1)(d+2)/2 mults, d(d+1)/2 adds.
 *   Sec. 4            one Newton step on truncated power series: evaluate and
 *                     differentiate the system at x(t) (algorithmic
 *                     differentiation), linearize into A(t) dx(t) = b(t) with
 *                     b = -f, factor A_0 (QR), forward-substitute degree by
 *                     degree: A_0 dx_k = b_k - sum_{j<k} A_{k-j} dx_j.
 *   Sec. 5            job decomposition: one job per polynomial for the
 *                     evaluation, one job per right-hand side update; jobs
 *                     never change a summation order, so the threaded run is
 *                     bit-identical to the serial one.
 *   Sec. 6            ||dx||: size of the update of the highest-degree coefficient.
 *
 * The md algorithms are not written out in the paper (it uses QDlib and
 * CAMPARY-generated code); the readings taken here are:
 *   TwoSum (Knuth), FastTwoSum (Dekker), TwoProd with fma.
 *   K = 2 add : AccurateDWPlusDW (Joldes-Muller-Popescu 2017), 8 adds, 12 subs.
 *   K = 2 mul : TwoProd(x0,y0) + (x0*y1 + x1*y0), then FastTwoSum (Hida-Li-Bailey).
 *   K >= 3    : level-by-level accumulation.  Level n < K holds the exact terms
 *               of order 2^(-53 n); they are summed by a TwoSum chain whose
 *               errors are carried to level n+1.  Level K is summed with plain
 *               additions.  Multiplication uses TwoProd for x_i*y_j with
 *               i+j <= K-1 and plain products for i+j = K.  The K+1 level sums
 *               are renormalised (bottom-up TwoSum sweep, then a top-down
 *               TwoSum sweep that skips zero errors) into K limbs.
 *   div       : long division with K+1 quotient limbs q_i = r_0 / y_0.
 *   sqrt      : hardware sqrt of the leading limb, then ceil(log2 K)+1 Heron
 *               steps s <- (s + a/s)/2 with exact halving.
 *   complex   : (a+bi)(c+di) = (ac - bd) + (ad + bc)i.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MAXK 10
#define MAXT 160
#define MAXV 4

/* ------------------------------------------------------------------ counts */
#ifdef ORACLE_COUNT
/* add, sub, mul, div, fma, sqrt, twoprod calls, series-level md mul, series-level md add, twosum calls */
long long orc_cnt[10];
static double oADD(double a, double b) { orc_cnt[0]++; return a + b; }
static double oSUB(double a, double b) { orc_cnt[1]++; return a - b; }
static double oMUL(double a, double b) { orc_cnt[2]++; return a * b; }
static double oDIV(double a, double b) { orc_cnt[3]++; return a / b; }
static double oFMA(double a, double b, double c) { orc_cnt[4]++; return fma(a, b, c); }
static double oSQRT(double a) { orc_cnt[5]++; return sqrt(a); }
#define CNT_TWOPROD() (orc_cnt[6]++)
#define CNT_SMUL() (orc_cnt[7]++)
#define CNT_SADD() (orc_cnt[8]++)
#define CNT_TWOSUM() (orc_cnt[9]++)
#else
long long orc_cnt[10];
#define oADD(a, b) ((a) + (b))
#define oSUB(a, b) ((a) - (b))
#define oMUL(a, b) ((a) * (b))
#define oDIV(a, b) ((a) / (b))
#define oFMA(a, b, c) fma((a), (b), (c))
#define oSQRT(a) sqrt(a)
#define CNT_TWOPROD() ((void)0)
#define CNT_SMUL() ((void)0)
#define CNT_SADD() ((void)0)
#define CNT_TWOSUM() ((void)0)
#endif

void orc_count_reset(void) { memset(orc_cnt, 0, sizeof(orc_cnt)); }
void orc_count_get(long long *out) { memcpy(out, orc_cnt, sizeof(orc_cnt)); }
int orc_is_counting(void) {
#ifdef ORACLE_COUNT
  return 1;
#else
  return 0;
#endif
}

/* --------------------------------------------- error-free transformations */
static void two_sum(double a, double b, double *s, double *e) {
  CNT_TWOSUM();
  double ss = oADD(a, b);
  double t = oSUB(ss, a);
  *e = oADD(oSUB(a, oSUB(ss, t)), oSUB(b, t));
  *s = ss;
}

static void fast_two_sum(double a, double b, double *s, double *e) {
  double ss = oADD(a, b);
  *e = oSUB(b, oSUB(ss, a));
  *s = ss;
}

static void two_prod(double a, double b, double *p, double *e) {
  double pp = oMUL(a, b);
  *e = oFMA(a, b, -pp);
  *p = pp;
  CNT_TWOPROD();
}

/* Renormalise m terms t[0..m-1] (roughly decreasing) into K limbs. */
static void renorm(const double *t, int m, int K, double *z) {
  double c[MAXT + 2];
  double s = t[m - 1];
  for (int i = m - 2; i >= 0; --i) two_sum(t[i], s, &s, &c[i + 1]);
  c[0] = s;
  int j = 0, i = 1;
  double e = c[0];
  for (; i < m && j < K - 1; ++i) {
    double r, f;
    two_sum(e, c[i], &r, &f);
    if (f != 0.0) {
      z[j++] = r;
      e = f;
    } else {
      e = r;
    }
  }
  for (; i < m; ++i) e = oADD(e, c[i]);
  z[j++] = e;
  for (; j < K; ++j) z[j] = 0.0;
}

/* ------------------------------------------------------------ md real ops */
static void md_add(int K, const double *x, const double *y, double *z) {
  if (K == 1) {
    z[0] = oADD(x[0], y[0]);
    return;
  }
  if (K == 2) { /* AccurateDWPlusDW */
    double sh, sl, th, tl, c, vh, vl, w, zh, zl;
    two_sum(x[0], y[0], &sh, &sl);
    two_sum(x[1], y[1], &th, &tl);
    c = oADD(sl, th);
    fast_two_sum(sh, c, &vh, &vl);
    w = oADD(tl, vl);
    fast_two_sum(vh, w, &zh, &zl);
    z[0] = zh;
    z[1] = zl;
    return;
  }
  double lv[MAXK + 1], carry[MAXT], nc[MAXT];
  int ncar = 0;
  for (int n = 0; n < K; ++n) {
    double s;
    int nn = 0;
    two_sum(x[n], y[n], &s, &nc[nn++]);
    for (int i = 0; i < ncar; ++i) two_sum(s, carry[i], &s, &nc[nn++]);
    lv[n] = s;
    memcpy(carry, nc, sizeof(double) * nn);
    ncar = nn;
  }
  double s = carry[0];
  for (int i = 1; i < ncar; ++i) s = oADD(s, carry[i]);
  lv[K] = s;
  renorm(lv, K + 1, K, z);
}

static void md_neg(int K, const double *x, double *z) {
  for (int i = 0; i < K; ++i) z[i] = -x[i];
}

static void md_sub(int K, const double *x, const double *y, double *z) {
  double ny[MAXK];
  md_neg(K, y, ny);
  md_add(K, x, ny, z);
}

static void md_mul(int K, const double *x, const double *y, double *z) {
  if (K == 1) {
    z[0] = oMUL(x[0], y[0]);
    return;
  }
  if (K == 2) {
    double p, e;
    two_prod(x[0], y[0], &p, &e);
    double t1 = oMUL(x[0], y[1]);
    double t2 = oMUL(x[1], y[0]);
    e = oADD(e, oADD(t1, t2));
    fast_two_sum(p, e, &z[0], &z[1]);
    return;
  }
  double lv[MAXK + 1], carry[MAXT], nc[MAXT], low[MAXK], nlow[MAXK], hi[MAXK];
  int ncar = 0, nl = 0;
  for (int n = 0; n < K; ++n) {
    for (int i = 0; i <= n; ++i) two_prod(x[i], y[n - i], &hi[i], &nlow[i]);
    double s = hi[0];
    int nn = 0;
    for (int i = 1; i <= n; ++i) two_sum(s, hi[i], &s, &nc[nn++]);
    for (int i = 0; i < nl; ++i) two_sum(s, low[i], &s, &nc[nn++]);
    for (int i = 0; i < ncar; ++i) two_sum(s, carry[i], &s, &nc[nn++]);
    lv[n] = s;
    memcpy(carry, nc, sizeof(double) * nn);
    ncar = nn;
    memcpy(low, nlow, sizeof(double) * (n + 1));
    nl = n + 1;
  }
  double s = oMUL(x[1], y[K - 1]);
  for (int i = 2; i <= K - 1; ++i) s = oADD(s, oMUL(x[i], y[K - i]));
  for (int i = 0; i < nl; ++i) s = oADD(s, low[i]);
  for (int i = 0; i < ncar; ++i) s = oADD(s, carry[i]);
  lv[K] = s;
  renorm(lv, K + 1, K, z);
}

/* md times double */
static void md_mul_d(int K, const double *x, double b, double *z) {
  if (K == 1) {
    z[0] = oMUL(x[0], b);
    return;
  }
  if (K == 2) {
    double p, e;
    two_prod(x[0], b, &p, &e);
    e = oADD(e, oMUL(x[1], b));
    fast_two_sum(p, e, &z[0], &z[1]);
    return;
  }
  double lv[MAXK + 1], carry[MAXT], nc[MAXT];
  int ncar = 0;
  double lo_prev = 0.0;
  for (int n = 0; n < K; ++n) {
    double h, l;
    two_prod(x[n], b, &h, &l);
    if (n == 0) {
      lv[0] = h;
    } else {
      double s = h;
      int nn = 0;
      two_sum(s, lo_prev, &s, &nc[nn++]);
      for (int i = 0; i < ncar; ++i) two_sum(s, carry[i], &s, &nc[nn++]);
      lv[n] = s;
      memcpy(carry, nc, sizeof(double) * nn);
      ncar = nn;
    }
    lo_prev = l;
  }
  double s = lo_prev;
  for (int i = 0; i < ncar; ++i) s = oADD(s, carry[i]);
  lv[K] = s;
  renorm(lv, K + 1, K, z);
}

static void md_div(int K, const double *x, const double *y, double *z) {
  if (K == 1) {
    z[0] = oDIV(x[0], y[0]);
    return;
  }
  double q[MAXK + 1], r[MAXK], t[MAXK];
  memcpy(r, x, sizeof(double) * K);
  for (int i = 0; i <= K; ++i) {
    q[i] = oDIV(r[0], y[0]);
    if (i < K) {
      md_mul_d(K, y, q[i], t);
      md_sub(K, r, t, r);
    }
  }
  renorm(q, K + 1, K, z);
}

static int sqrt_iters(int K) {
  int l = 0;
  while ((1 << l) < K) ++l;
  return l + 1;
}

static void md_sqrt(int K, const double *a, double *z) {
  if (K == 1) {
    z[0] = oSQRT(a[0]);
    return;
  }
  if (a[0] == 0.0) {
    for (int i = 0; i < K; ++i) z[i] = 0.0;
    return;
  }
  double s[MAXK], t[MAXK];
  s[0] = oSQRT(a[0]);
  for (int i = 1; i < K; ++i) s[i] = 0.0;
  int it = sqrt_iters(K);
  for (int k = 0; k < it; ++k) {
    md_div(K, a, s, t);
    md_add(K, s, t, s);
    for (int i = 0; i < K; ++i) s[i] = oMUL(s[i], 0.5);
  }
  memcpy(z, s, sizeof(double) * K);
}

/* --------------------------------------------------------- md complex ops */
typedef struct {
  double v[2][MAXK];
} mdc;

static void c_zero(mdc *z) { memset(z, 0, sizeof(*z)); }

static void c_add(int K, int P, const mdc *a, const mdc *b, mdc *z) {
  CNT_SADD();
  for (int p = 0; p < P; ++p) md_add(K, a->v[p], b->v[p], z->v[p]);
}

static void c_sub(int K, int P, const mdc *a, const mdc *b, mdc *z) {
  CNT_SADD();
  for (int p = 0; p < P; ++p) md_sub(K, a->v[p], b->v[p], z->v[p]);
}

static void c_mul(int K, int P, const mdc *a, const mdc *b, mdc *z) {
  CNT_SMUL();
  if (P == 1) {
    md_mul(K, a->v[0], b->v[0], z->v[0]);
    return;
  }
  double ac[MAXK], bd[MAXK], ad[MAXK], bc[MAXK];
  md_mul(K, a->v[0], b->v[0], ac);
  md_mul(K, a->v[1], b->v[1], bd);
  md_mul(K, a->v[0], b->v[1], ad);
  md_mul(K, a->v[1], b->v[0], bc);
  md_sub(K, ac, bd, z->v[0]);
  md_add(K, ad, bc, z->v[1]);
}

/* complex times md real */
static void c_mul_real(int K, int P, const mdc *a, const double *r, mdc *z) {
  for (int p = 0; p < P; ++p) md_mul(K, a->v[p], r, z->v[p]);
}

static void c_mul_d(int K, int P, const mdc *a, double b, mdc *z) {
  for (int p = 0; p < P; ++p) md_mul_d(K, a->v[p], b, z->v[p]);
}

static void c_conj(int K, int P, const mdc *a, mdc *z) {
  *z = *a;
  if (P == 2) md_neg(K, a->v[1], z->v[1]);
}

static void c_abs2(int K, int P, const mdc *a, double *z) {
  if (P == 1) {
    md_mul(K, a->v[0], a->v[0], z);
    return;
  }
  double t1[MAXK], t2[MAXK];
  md_mul(K, a->v[0], a->v[0], t1);
  md_mul(K, a->v[1], a->v[1], t2);
  md_add(K, t1, t2, z);
}

static void c_div(int K, int P, const mdc *a, const mdc *b, mdc *z) {
  if (P == 1) {
    md_div(K, a->v[0], b->v[0], z->v[0]);
    return;
  }
  double cc[MAXK], dd[MAXK], den[MAXK], t1[MAXK], t2[MAXK], nr[MAXK], ni[MAXK];
  md_mul(K, b->v[0], b->v[0], cc);
  md_mul(K, b->v[1], b->v[1], dd);
  md_add(K, cc, dd, den);
  md_mul(K, a->v[0], b->v[0], t1);
  md_mul(K, a->v[1], b->v[1], t2);
  md_add(K, t1, t2, nr);
  md_mul(K, a->v[1], b->v[0], t1);
  md_mul(K, a->v[0], b->v[1], t2);
  md_sub(K, t1, t2, ni);
  md_div(K, nr, den, z->v[0]);
  md_div(K, ni, den, z->v[1]);
}

/* ------------------------------------------------------- layout helpers */
/* series vector [P][K][n][d+1] <-> mdc s[j*(d+1)+k] */
static void load_series(int K, int P, int n, int d, const double *x, mdc *s) {
  long D1 = d + 1;
  for (int j = 0; j < n; ++j)
    for (int k = 0; k <= d; ++k) {
      mdc *z = &s[j * D1 + k];
      c_zero(z);
      for (int p = 0; p < P; ++p)
        for (int l = 0; l < K; ++l) z->v[p][l] = x[(((long)p * K + l) * n + j) * D1 + k];
    }
}

static void store_series(int K, int P, int n, int d, const mdc *s, double *x) {
  long D1 = d + 1;
  for (int j = 0; j < n; ++j)
    for (int k = 0; k <= d; ++k)
      for (int p = 0; p < P; ++p)
        for (int l = 0; l < K; ++l) x[(((long)p * K + l) * n + j) * D1 + k] = s[j * D1 + k].v[p][l];
}

/* matrix series [P][K][d+1][col][row] <-> mdc a[(k*n + row)*n + col] */
/* matrix series: API [P][K][d+1][n columns][N rows] <-> a[(k*N + r)*n + c] */
static void load_mats(int K, int P, int N, int n, int d, const double *A, mdc *a) {
  long nn = (long)N * n;
  for (int k = 0; k <= d; ++k)
    for (int r = 0; r < N; ++r)
      for (int c = 0; c < n; ++c) {
        mdc *z = &a[(k * (long)N + r) * n + c];
        c_zero(z);
        for (int p = 0; p < P; ++p)
          for (int l = 0; l < K; ++l) z->v[p][l] = A[(((long)p * K + l) * (d + 1) + k) * nn + (long)c * N + r];
      }
}

static void store_mats(int K, int P, int N, int n, int d, const mdc *a, double *A) {
  long nn = (long)N * n;
  for (int k = 0; k <= d; ++k)
    for (int r = 0; r < N; ++r)
      for (int c = 0; c < n; ++c)
        for (int p = 0; p < P; ++p)
          for (int l = 0; l < K; ++l)
            A[(((long)p * K + l) * (d + 1) + k) * nn + (long)c * N + r] = a[(k * (long)N + r) * n + c].v[p][l];
}

/* ------------------------------------------------------------ series ops */
/* z = x * y truncated at degree d (Sec. 3): z_k = sum_{i=0..k} x_i y_{k-i} */
static void s_conv(int K, int P, int d, const mdc *x, const mdc *y, mdc *z) {
  for (int k = 0; k <= d; ++k) {
    mdc acc, t;
    c_mul(K, P, &x[0], &y[k], &acc);
    for (int i = 1; i <= k; ++i) {
      c_mul(K, P, &x[i], &y[k - i], &t);
      c_add(K, P, &acc, &t, &acc);
    }
    z[k] = acc;
  }
}

int orc_md_op(int op, int K, int cplx, long count, const double *x, const double *y, double *z) {
  /* op: 0 add, 1 sub, 2 mul, 3 div, 4 sqrt (real), 5 mul by double (y: [count]) ;
     layout [P][K][count] */
  int P = cplx ? 2 : 1;
  if (K < 1 || K > MAXK) return 1;
  if (op == 4 && cplx) return 1;
  for (long i = 0; i < count; ++i) {
    mdc a, b, c;
    c_zero(&a);
    c_zero(&b);
    for (int p = 0; p < P; ++p)
      for (int l = 0; l < K; ++l) {
        a.v[p][l] = x[((long)p * K + l) * count + i];
        if (op <= 3) b.v[p][l] = y[((long)p * K + l) * count + i];
      }
    switch (op) {
      case 0: c_add(K, P, &a, &b, &c); break;
      case 1: c_sub(K, P, &a, &b, &c); break;
      case 2: c_mul(K, P, &a, &b, &c); break;
      case 3: c_div(K, P, &a, &b, &c); break;
      case 4: md_sqrt(K, a.v[0], c.v[0]); break;
      case 5: c_mul_d(K, P, &a, y[i], &c); break;
      default: return 1;
    }
    for (int p = 0; p < P; ++p)
      for (int l = 0; l < K; ++l) z[((long)p * K + l) * count + i] = c.v[p][l];
  }
  return 0;
}

int orc_series_conv(int K, int cplx, int d, long count, const double *x, const double *y, double *z) {
  /* count independent products, layout [P][K][count][d+1] */
  int P = cplx ? 2 : 1;
  mdc *xs = malloc(sizeof(mdc) * count * (d + 1));
  mdc *ys = malloc(sizeof(mdc) * count * (d + 1));
  mdc *zs = malloc(sizeof(mdc) * count * (d + 1));
  load_series(K, P, (int)count, d, x, xs);
  load_series(K, P, (int)count, d, y, ys);
  for (long c = 0; c < count; ++c) s_conv(K, P, d, xs + c * (d + 1), ys + c * (d + 1), zs + c * (d + 1));
  store_series(K, P, (int)count, d, zs, z);
  free(xs);
  free(ys);
  free(zs);
  return 0;
}

/* ---------------------------------------------- evaluate and differentiate */
/*
 * One monomial c * prod_q x_{j_q}^{a_q} * t^{a_t} at the series x(t)
 * (Sec. 4; algorithmic differentiation in the sense of Griewank-Walther):
 *   common factor F = prod_q x_{j_q}^{a_q - 1}  (repeated products, variable order),
 *   Speelpenning product of the m distinct variables: forward products
 *   p_q = p_{q-1} x_{j_q}, backward products s_q = x_{j_q} s_{q+1}, and cross
 *   products p_{q-1} s_{q+1}, giving the value P = p_m and the m partials,
 *   G = F P, D_q = F * partial_q, value = c G, derivative q = (a_q c) D_q,
 *   both shifted by a_t powers of t (t has the fixed series 0 + 1 t).
 * Series marked "unit" are the constant 1 and are never multiplied.
 */
typedef struct {
  int K, P, d;
  mdc *buf; /* scratch: (2*MAXV + 4) series */
} evctx;

static void conv_or_copy(int K, int P, int d, const mdc *x, int xunit, const mdc *y, int yunit, mdc *z, int *zunit) {
  if (xunit && yunit) {
    *zunit = 1;
    return;
  }
  *zunit = 0;
  if (xunit) {
    memcpy(z, y, sizeof(mdc) * (d + 1));
  } else if (yunit) {
    memcpy(z, x, sizeof(mdc) * (d + 1));
  } else {
    s_conv(K, P, d, x, y, z);
  }
}

/* Returns m (number of x-variables); writes value series V, partial series
   Dq[q] (for q < m, variable vj[q]); all already scaled and shifted. */
static int eval_monomial(evctx *cx, int n, int nv, const int *idx, const int *expo, const mdc *coef, const mdc *xs,
                         mdc *V, mdc *Dq, int *vj) {
  int K = cx->K, P = cx->P, d = cx->d;
  long D1 = d + 1;
  int m = 0, at = 0, va[MAXV];
  for (int q = 0; q < nv; ++q) {
    if (idx[q] == n) {
      at = expo[q];
    } else {
      vj[m] = idx[q];
      va[m] = expo[q];
      ++m;
    }
  }
  mdc *F = cx->buf;
  mdc *T = F + D1;          /* temp */
  mdc *pf = T + D1;         /* forward products p_1..p_m: MAXV series */
  mdc *sb = pf + MAXV * D1; /* backward products: MAXV series */
  mdc *G = sb + MAXV * D1;
  mdc *Dt = G + D1;
  int Funit = 1, tmpu;
  /* common factor */
  for (int q = 0; q < m; ++q)
    for (int e = 1; e < va[q]; ++e) {
      if (Funit) {
        memcpy(F, xs + (long)vj[q] * D1, sizeof(mdc) * D1);
        Funit = 0;
      } else {
        s_conv(K, P, d, F, xs + (long)vj[q] * D1, T);
        memcpy(F, T, sizeof(mdc) * D1);
      }
    }
  /* Speelpenning products */
  const mdc *P_ser = NULL;
  int Punit = 1;
  if (m >= 1) {
    /* forward: pf[q] = p_{q+1} = x_{j_0} ... x_{j_q}; pf[0] aliases x_{j_0} */
    for (int q = 1; q < m; ++q) {
      const mdc *prev = (q == 1) ? xs + (long)vj[0] * D1 : pf + (long)(q - 1) * D1;
      s_conv(K, P, d, prev, xs + (long)vj[q] * D1, pf + (long)q * D1);
    }
    /* backward: sb[q] = x_{j_q} ... x_{j_{m-1}}; sb[m-1] aliases x_{j_{m-1}} */
    for (int q = m - 2; q >= 1; --q) {
      const mdc *next = (q == m - 2) ? xs + (long)vj[m - 1] * D1 : sb + (long)(q + 1) * D1;
      s_conv(K, P, d, xs + (long)vj[q] * D1, next, sb + (long)q * D1);
    }
    P_ser = (m == 1) ? xs + (long)vj[0] * D1 : pf + (long)(m - 1) * D1;
    Punit = 0;
  }
  /* value: G = F * P, V = c G shifted by at */
  int Gunit;
  conv_or_copy(K, P, d, F, Funit, P_ser, Punit, G, &Gunit);
  for (int k = 0; k <= d; ++k) {
    c_zero(&V[k]);
    if (k < at) continue;
    if (Gunit) {
      if (k == at) V[k] = *coef;
    } else {
      c_mul(K, P, coef, &G[k - at], &V[k]);
    }
  }
  /* partials */
  for (int q = 0; q < m; ++q) {
    const mdc *dser;
    int dunit;
    if (m == 1) {
      dser = NULL;
      dunit = 1;
    } else if (q == 0) {
      dser = (m == 2) ? xs + (long)vj[1] * D1 : sb + 1 * D1;
      dunit = 0;
    } else if (q == m - 1) {
      dser = (m == 2) ? xs + (long)vj[0] * D1 : pf + (long)(m - 2) * D1;
      dunit = 0;
    } else {
      const mdc *left = (q == 1) ? xs + (long)vj[0] * D1 : pf + (long)(q - 1) * D1;
      const mdc *right = (q == m - 2) ? xs + (long)vj[m - 1] * D1 : sb + (long)(q + 1) * D1;
      s_conv(K, P, d, left, right, T);
      dser = T;
      dunit = 0;
    }
    conv_or_copy(K, P, d, F, Funit, dser, dunit, Dt, &tmpu);
    mdc cq;
    if (va[q] == 1)
      cq = *coef;
    else
      c_mul_d(K, P, coef, (double)va[q], &cq);
    mdc *out = Dq + (long)q * D1;
    for (int k = 0; k <= d; ++k) {
      c_zero(&out[k]);
      if (k < at) continue;
      if (tmpu) {
        if (k == at) out[k] = cq;
      } else {
        c_mul(K, P, &cq, &Dt[k - at], &out[k]);
      }
    }
  }
  return m;
}

/* f_i = cst_i + sum_mono value; A_k[i][j] = sum_mono (d/dx_j value)_k, in CSR order */
static void eval_diff_internal(int K, int P, int N, int n, int d, const int *poly_ptr, const int *nvar,
                               const int *idx, const int *expo, const mdc *coefs, const mdc *csts, const mdc *xs,
                               mdc *fs, mdc *as) {
  long D1 = d + 1;
  long nn = (long)N * n;
  for (long e = 0; e < D1 * nn; ++e) c_zero(&as[e]);
#pragma omp parallel
  {
    evctx cx;
    cx.K = K;
    cx.P = P;
    cx.d = d;
    cx.buf = malloc(sizeof(mdc) * D1 * (2 * MAXV + 4));
    mdc *V = malloc(sizeof(mdc) * D1);
    mdc *Dq = malloc(sizeof(mdc) * D1 * MAXV);
#pragma omp for schedule(dynamic, 1)
    for (int i = 0; i < N; ++i) {
      mdc *f = fs + (long)i * D1;
      for (int k = 0; k <= d; ++k) c_zero(&f[k]);
      f[0] = csts[i];
      for (int mo = poly_ptr[i]; mo < poly_ptr[i + 1]; ++mo) {
        int vj[MAXV];
        int m = eval_monomial(&cx, n, nvar[mo], idx + (long)mo * MAXV, expo + (long)mo * MAXV, &coefs[mo], xs, V, Dq, vj);
        for (int k = 0; k <= d; ++k) c_add(K, P, &f[k], &V[k], &f[k]);
        for (int q = 0; q < m; ++q)
          for (int k = 0; k <= d; ++k) {
            mdc *a = &as[(k * (long)N + i) * n + vj[q]];
            c_add(K, P, a, &Dq[(long)q * D1 + k], a);
          }
      }
    }
    free(cx.buf);
    free(V);
    free(Dq);
  }
}

static void load_scalars(int K, int P, long count, const double *src, mdc *dst) {
  for (long m = 0; m < count; ++m) {
    c_zero(&dst[m]);
    for (int p = 0; p < P; ++p)
      for (int l = 0; l < K; ++l) dst[m].v[p][l] = src[((long)p * K + l) * count + m];
  }
}

/* N polynomials (N >= n) in n unknowns; variable n is t */
static int check_system(int K, int N, int n, int d, int nmono, const int *poly_ptr, const int *nvar, const int *idx,
                        const int *expo) {
  if (K < 1 || K > MAXK || n < 1 || N < n || d < 0) return 1;
  if (poly_ptr[0] != 0 || poly_ptr[N] != nmono) return 1;
  for (int i = 0; i < N; ++i)
    if (poly_ptr[i + 1] < poly_ptr[i]) return 1;
  for (int m = 0; m < nmono; ++m) {
    if (nvar[m] < 0 || nvar[m] > MAXV) return 1;
    for (int q = 0; q < nvar[m]; ++q) {
      int v = idx[(long)m * MAXV + q], e = expo[(long)m * MAXV + q];
      if (v < 0 || v > n || e < 1) return 1;
      for (int q2 = 0; q2 < q; ++q2)
        if (idx[(long)m * MAXV + q2] == v) return 1;
    }
  }
  return 0;
}

/* f: [P][K][N][d+1], A: [P][K][d+1][n][N] */
int orc_eval_diff_ls(int K, int cplx, int N, int n, int d, int nmono, const int *poly_ptr, const int *nvar,
                     const int *idx, const int *expo, const double *coef, const double *cst, const double *x, double *f,
                     double *A) {
  int P = cplx ? 2 : 1;
  if (check_system(K, N, n, d, nmono, poly_ptr, nvar, idx, expo)) return 1;
  long D1 = d + 1;
  mdc *coefs = malloc(sizeof(mdc) * (nmono > 0 ? nmono : 1));
  mdc *csts = malloc(sizeof(mdc) * N);
  mdc *xs = malloc(sizeof(mdc) * n * D1);
  mdc *fs = malloc(sizeof(mdc) * N * D1);
  mdc *as = malloc(sizeof(mdc) * D1 * N * n);
  load_scalars(K, P, nmono, coef, coefs);
  load_scalars(K, P, N, cst, csts);
  load_series(K, P, n, d, x, xs);
  eval_diff_internal(K, P, N, n, d, poly_ptr, nvar, idx, expo, coefs, csts, xs, fs, as);
  store_series(K, P, N, d, fs, f);
  store_mats(K, P, N, n, d, as, A);
  free(coefs);
  free(csts);
  free(xs);
  free(fs);
  free(as);
  return 0;
}

int orc_eval_diff(int K, int cplx, int n, int d, int nmono, const int *poly_ptr, const int *nvar, const int *idx,
                  const int *expo, const double *coef, const double *cst, const double *x, double *f, double *A) {
  return orc_eval_diff_ls(K, cplx, n, n, d, nmono, poly_ptr, nvar, idx, expo, coef, cst, x, f, A);
}

/* ------------------------------------------------ Householder QR of A_0 */
/*
 * Golub-Van Loan Householder QR of the N x n matrix A_0 (N >= n; Sec. 4:
 * least squares for N > n), complex form.  Column j: x = a[j:N, j],
 * alpha = ||x||_2, phase e = x_0/|x_0| (1 if x_0 = 0), v = x + e alpha e_1,
 * beta = 2/(v^H v) = 1/(alpha (alpha + |x_0|)), R_jj = -e alpha; the trailing
 * columns get a_c -= beta (v^H a_c) v.  v_0 is kept in vd[j], v_i (i > j) stays
 * below the diagonal, R above it.  Returns 4 when alpha = 0 (singular A_0).
 */
typedef struct {
  int K, P, N, n;
  mdc *a;    /* row-major N x n: a[r*n + c] */
  mdc *vd;   /* [n] v_0 of each reflector */
  mdc *rd;   /* [n] R_jj */
  double (*beta)[MAXK]; /* [n] */
} qrf;

static int qr_factor(qrf *q) {
  int K = q->K, P = q->P, N = q->N, n = q->n;
  mdc *a = q->a;
  for (int j = 0; j < n; ++j) {
    double ss[MAXK], t[MAXK], alpha[MAXK], a0[MAXK], s2[MAXK];
    c_abs2(K, P, &a[(long)j * n + j], ss);
    for (int i = j + 1; i < N; ++i) {
      c_abs2(K, P, &a[(long)i * n + j], t);
      md_add(K, ss, t, ss);
    }
    md_sqrt(K, ss, alpha);
    if (alpha[0] == 0.0) return 4;
    mdc x0 = a[(long)j * n + j], ph;
    c_zero(&ph);
    if (P == 1) {
      for (int l = 0; l < K; ++l) a0[l] = (x0.v[0][0] < 0.0) ? -x0.v[0][l] : x0.v[0][l];
      ph.v[0][0] = (x0.v[0][0] < 0.0) ? -1.0 : 1.0;
    } else {
      c_abs2(K, P, &x0, s2);
      md_sqrt(K, s2, a0);
      if (a0[0] == 0.0) {
        ph.v[0][0] = 1.0;
      } else {
        md_div(K, x0.v[0], a0, ph.v[0]);
        md_div(K, x0.v[1], a0, ph.v[1]);
      }
    }
    mdc pa, v0, rjj;
    c_mul_real(K, P, &ph, alpha, &pa);
    c_add(K, P, &x0, &pa, &v0);
    for (int p = 0; p < P; ++p) md_neg(K, pa.v[p], rjj.v[p]);
    if (P == 1) memset(rjj.v[1], 0, sizeof(rjj.v[1]));
    double den[MAXK], one[MAXK], beta[MAXK];
    md_add(K, alpha, a0, t);
    md_mul(K, alpha, t, den);
    memset(one, 0, sizeof(one));
    one[0] = 1.0;
    md_div(K, one, den, beta);
    q->vd[j] = v0;
    q->rd[j] = rjj;
    memcpy(q->beta[j], beta, sizeof(double) * MAXK);
    for (int c = j + 1; c < n; ++c) {
      mdc w, tt, cv, tau;
      c_conj(K, P, &v0, &cv);
      c_mul(K, P, &cv, &a[(long)j * n + c], &w);
      for (int i = j + 1; i < N; ++i) {
        c_conj(K, P, &a[(long)i * n + j], &cv);
        c_mul(K, P, &cv, &a[(long)i * n + c], &tt);
        c_add(K, P, &w, &tt, &w);
      }
      c_mul_real(K, P, &w, beta, &tau);
      c_mul(K, P, &tau, &v0, &tt);
      c_sub(K, P, &a[(long)j * n + c], &tt, &a[(long)j * n + c]);
      for (int i = j + 1; i < N; ++i) {
        c_mul(K, P, &tau, &a[(long)i * n + j], &tt);
        c_sub(K, P, &a[(long)i * n + c], &tt, &a[(long)i * n + c]);
      }
    }
  }
  return 0;
}

/* y <- Q^H y = H_{n-1} ... H_0 y (y has N entries) */
static void qr_apply_qh(qrf *q, mdc *y) {
  int K = q->K, P = q->P, N = q->N, n = q->n;
  for (int j = 0; j < n; ++j) {
    mdc w, tt, cv, tau;
    c_conj(K, P, &q->vd[j], &cv);
    c_mul(K, P, &cv, &y[j], &w);
    for (int i = j + 1; i < N; ++i) {
      c_conj(K, P, &q->a[(long)i * n + j], &cv);
      c_mul(K, P, &cv, &y[i], &tt);
      c_add(K, P, &w, &tt, &w);
    }
    c_mul_real(K, P, &w, q->beta[j], &tau);
    c_mul(K, P, &tau, &q->vd[j], &tt);
    c_sub(K, P, &y[j], &tt, &y[j]);
    for (int i = j + 1; i < N; ++i) {
      c_mul(K, P, &tau, &q->a[(long)i * n + j], &tt);
      c_sub(K, P, &y[i], &tt, &y[i]);
    }
  }
}

/* column-oriented back substitution R x = y[0:n] with the top n x n block R
   (y is overwritten) */
static void qr_backsub(qrf *q, mdc *y, mdc *x) {
  int K = q->K, P = q->P, n = q->n;
  for (int c = n - 1; c >= 0; --c) {
    c_div(K, P, &y[c], &q->rd[c], &x[c]);
    for (int i = 0; i < c; ++i) {
      mdc tt;
      c_mul(K, P, &q->a[(long)i * n + c], &x[c], &tt);
      c_sub(K, P, &y[i], &tt, &y[i]);
    }
  }
}

/* ------------------------------------------------------------ LU (N = n) */
/*
 * Gaussian elimination with partial pivoting (Sec. 4: when N = n an LU
 * factorization can be applied; Golub-Van Loan, Alg. 3.4.1).  Column j: the
 * pivot is the first row i >= j of largest |re| + |im| of the leading limbs;
 * rows j and p are swapped; the multipliers a_ij * (1/a_jj) are stored below
 * the diagonal; the trailing entries get a_ik -= l_ij a_jk.  Returns 4 when a
 * pivot is zero (singular A_0).
 */
typedef struct {
  int K, P, n;
  mdc *a;   /* row-major n x n */
  int *piv; /* [n] row swapped with row j at step j */
} luf;

static double cabs1_lead(int P, const mdc *z) { return fabs(z->v[0][0]) + (P == 2 ? fabs(z->v[1][0]) : 0.0); }

static int lu_factor(luf *f) {
  int K = f->K, P = f->P, n = f->n;
  mdc *a = f->a;
  for (int j = 0; j < n; ++j) {
    int p = j;
    double best = cabs1_lead(P, &a[(long)j * n + j]);
    for (int i = j + 1; i < n; ++i) {
      double v = cabs1_lead(P, &a[(long)i * n + j]);
      if (v > best) {
        best = v;
        p = i;
      }
    }
    if (!(best > 0.0)) return 4;
    f->piv[j] = p;
    if (p != j)
      for (int c = 0; c < n; ++c) {
        mdc t = a[(long)j * n + c];
        a[(long)j * n + c] = a[(long)p * n + c];
        a[(long)p * n + c] = t;
      }
    mdc one, ri;
    c_zero(&one);
    one.v[0][0] = 1.0;
    c_div(K, P, &one, &a[(long)j * n + j], &ri);
    for (int i = j + 1; i < n; ++i) {
      c_mul(K, P, &a[(long)i * n + j], &ri, &a[(long)i * n + j]);
      for (int c = j + 1; c < n; ++c) {
        mdc tt;
        c_mul(K, P, &a[(long)i * n + j], &a[(long)j * n + c], &tt);
        c_sub(K, P, &a[(long)i * n + c], &tt, &a[(long)i * n + c]);
      }
    }
  }
  return 0;
}

/* A_0 x = y by P, L (unit, forward) and U (backward, row by row, dividing by
   u_jj); y is overwritten */
static void lu_solve(const luf *f, mdc *y, mdc *x) {
  int K = f->K, P = f->P, n = f->n;
  const mdc *a = f->a;
  for (int j = 0; j < n; ++j)
    if (f->piv[j] != j) {
      mdc t = y[j];
      y[j] = y[f->piv[j]];
      y[f->piv[j]] = t;
    }
  for (int i = 1; i < n; ++i)
    for (int j = 0; j < i; ++j) {
      mdc tt;
      c_mul(K, P, &a[(long)i * n + j], &y[j], &tt);
      c_sub(K, P, &y[i], &tt, &y[i]);
    }
  for (int i = n - 1; i >= 0; --i) {
    mdc s = y[i];
    for (int j = i + 1; j < n; ++j) {
      mdc tt;
      c_mul(K, P, &a[(long)i * n + j], &x[j], &tt);
      c_sub(K, P, &s, &tt, &s);
    }
    c_div(K, P, &s, &a[(long)i * n + i], &x[i]);
  }
}

/* A_0 factored by QR (method 0) or LU (method 1); solve A_0 x = y */
typedef struct {
  int method;
  qrf q;
  luf l;
} fact;

static int fact_init(fact *f, int method, int K, int P, int N, int n, const mdc *a0) {
  long nn = (long)N * n;
  memset(f, 0, sizeof(*f));
  f->method = method;
  if (method == 1) {
    if (N != n) return 1; /* LU is for square A_0 */
    f->l.K = K;
    f->l.P = P;
    f->l.n = n;
    f->l.a = malloc(sizeof(mdc) * nn);
    f->l.piv = malloc(sizeof(int) * n);
    memcpy(f->l.a, a0, sizeof(mdc) * nn);
    return lu_factor(&f->l);
  }
  f->q.K = K;
  f->q.P = P;
  f->q.N = N;
  f->q.n = n;
  f->q.a = malloc(sizeof(mdc) * nn);
  f->q.vd = malloc(sizeof(mdc) * n);
  f->q.rd = malloc(sizeof(mdc) * n);
  f->q.beta = malloc(sizeof(double) * MAXK * n);
  memcpy(f->q.a, a0, sizeof(mdc) * nn);
  return qr_factor(&f->q);
}

/* x (n entries) solves A_0 x = r (N entries) exactly (N = n) or in the least
   squares sense (N > n, QR only) */
static void fact_solve(fact *f, const mdc *r, mdc *x) {
  int N = f->method == 1 ? f->l.n : f->q.N;
  mdc *y = malloc(sizeof(mdc) * N);
  memcpy(y, r, sizeof(mdc) * N);
  if (f->method == 1) {
    lu_solve(&f->l, y, x);
  } else {
    qr_apply_qh(&f->q, y);
    qr_backsub(&f->q, y, x);
  }
  free(y);
}

static void fact_free(fact *f) {
  free(f->l.a);
  free(f->l.piv);
  free(f->q.a);
  free(f->q.vd);
  free(f->q.rd);
  free(f->q.beta);
}

/*
 * Lower triangular block Toeplitz forward substitution (Sec. 4):
 *   r_k = b_k - A_k dx_0 - A_{k-1} dx_1 - ... - A_1 dx_{k-1}   (j ascending)
 *   A_0 dx_k = r_k  via  dx_k = R^{-1} Q^H r_k.
 * Each A_i dx_j is a dot product per row, summed over columns in ascending
 * order starting from the first product.  After dx_j is known, the job
 * "update r_k with A_{k-j} dx_j" runs for every k > j (Sec. 5); each job
 * touches one r_k only, so the parallel loop keeps the serial order.
 * as: [(k*n + row)*n + col]; bs, dxs: [k*n + i].
 */
static int linsolve_internal(int K, int P, int N, int n, int d, mdc *as, const mdc *bs, mdc *dxs,
                             double *rdiag_abs, int method) {
  long nn = (long)N * n;
  fact f;
  int st = fact_init(&f, method, K, P, N, n, as);
  if (st) {
    fact_free(&f);
    return st;
  }
  if (rdiag_abs)
    for (int i = 0; i < n; ++i) {
      const mdc *rd = method == 1 ? &f.l.a[(long)i * n + i] : &f.q.rd[i];
      double re = rd->v[0][0], im = (P == 2) ? rd->v[1][0] : 0.0;
      rdiag_abs[i] = sqrt(re * re + im * im);
    }
  mdc *r = malloc(sizeof(mdc) * (d + 1) * N);
  memcpy(r, bs, sizeof(mdc) * (d + 1) * N);
  for (int k = 0; k <= d; ++k) {
    fact_solve(&f, r + (long)k * N, dxs + (long)k * n);
    /* jobs: r_m -= A_{m-k} dx_k for every m > k */
#pragma omp parallel for schedule(dynamic, 1)
    for (int m = k + 1; m <= d; ++m) {
      const mdc *Am = as + (long)(m - k) * nn;
      const mdc *dx = dxs + (long)k * n;
      mdc *rm = r + (long)m * N;
      for (int row = 0; row < N; ++row) {
        mdc acc, tt;
        c_mul(K, P, &Am[(long)row * n + 0], &dx[0], &acc);
        for (int col = 1; col < n; ++col) {
          c_mul(K, P, &Am[(long)row * n + col], &dx[col], &tt);
          c_add(K, P, &acc, &tt, &acc);
        }
        c_sub(K, P, &rm[row], &acc, &rm[row]);
      }
    }
  }
  free(r);
  fact_free(&f);
  return 0;
}

/* vectors [P][K][n][d+1] <-> mdc v[k*n + i] (degree-major) */
static void load_vec_dm(int K, int P, int n, int d, const double *x, mdc *v) {
  long D1 = d + 1;
  for (int k = 0; k <= d; ++k)
    for (int i = 0; i < n; ++i) {
      mdc *z = &v[(long)k * n + i];
      c_zero(z);
      for (int p = 0; p < P; ++p)
        for (int l = 0; l < K; ++l) z->v[p][l] = x[(((long)p * K + l) * n + i) * D1 + k];
    }
}

static void store_vec_dm(int K, int P, int n, int d, const mdc *v, double *x) {
  long D1 = d + 1;
  for (int k = 0; k <= d; ++k)
    for (int i = 0; i < n; ++i)
      for (int p = 0; p < P; ++p)
        for (int l = 0; l < K; ++l) x[(((long)p * K + l) * n + i) * D1 + k] = v[(long)k * n + i].v[p][l];
}

/* A: [P][K][d+1][n][N], b: [P][K][N][d+1] -> dx: [P][K][n][d+1] */
int orc_lstsq(int K, int cplx, int N, int n, int d, const double *A, const double *b, double *dx, double *rdiag_abs,
              int method) {
  int P = cplx ? 2 : 1;
  if (K < 1 || K > MAXK || n < 1 || N < n || d < 0) return 1;
  long nn = (long)N * n;
  mdc *as = malloc(sizeof(mdc) * (d + 1) * nn);
  mdc *bs = malloc(sizeof(mdc) * (d + 1) * N);
  mdc *dxs = malloc(sizeof(mdc) * (d + 1) * n);
  load_mats(K, P, N, n, d, A, as);
  load_vec_dm(K, P, N, d, b, bs);
  int st = linsolve_internal(K, P, N, n, d, as, bs, dxs, rdiag_abs, method);
  if (!st) store_vec_dm(K, P, n, d, dxs, dx);
  free(as);
  free(bs);
  free(dxs);
  return st;
}

int orc_linsolve_m(int K, int cplx, int n, int d, const double *A, const double *b, double *dx, double *rdiag_abs,
                   int method) {
  return orc_lstsq(K, cplx, n, n, d, A, b, dx, rdiag_abs, method);
}

int orc_linsolve(int K, int cplx, int n, int d, const double *A, const double *b, double *dx, double *rdiag_abs) {
  return orc_linsolve_m(K, cplx, n, d, A, b, dx, rdiag_abs, 0);
}

/* ------------------------------------------------------ one Newton step */
/*
 * x <- x + dx with A(t) dx(t) = -f(x(t)) (Sec. 4).  dxnorm[0] = max_i |dx_{d,i}|
 * (size of the update of the highest-degree coefficient, Sec. 6, from the leading
 * limbs), dxnorm[1] = max over all coefficients of |dx_{k,i}|.
 */
/* N >= n polynomials; the linear systems are solved in the least squares
   sense when N > n (Sec. 4) */
int orc_newton_step_ls(int K, int cplx, int N, int n, int d, int nmono, const int *poly_ptr, const int *nvar,
                       const int *idx, const int *expo, const double *coef, const double *cst, double *x,
                       double *dxnorm, double *rdiag_abs, int method) {
  int P = cplx ? 2 : 1;
  if (check_system(K, N, n, d, nmono, poly_ptr, nvar, idx, expo)) return 1;
  long D1 = d + 1, nn = (long)N * n;
  mdc *coefs = malloc(sizeof(mdc) * (nmono > 0 ? nmono : 1));
  mdc *csts = malloc(sizeof(mdc) * N);
  mdc *xs = malloc(sizeof(mdc) * n * D1);
  mdc *fs = malloc(sizeof(mdc) * N * D1);
  mdc *as = malloc(sizeof(mdc) * D1 * nn);
  mdc *bs = malloc(sizeof(mdc) * D1 * N);
  mdc *dxs = malloc(sizeof(mdc) * D1 * n);
  load_scalars(K, P, nmono, coef, coefs);
  load_scalars(K, P, N, cst, csts);
  load_series(K, P, n, d, x, xs);
  eval_diff_internal(K, P, N, n, d, poly_ptr, nvar, idx, expo, coefs, csts, xs, fs, as);
  for (int k = 0; k <= d; ++k)
    for (int i = 0; i < N; ++i) {
      mdc *z = &bs[(long)k * N + i];
      for (int p = 0; p < P; ++p) md_neg(K, fs[(long)i * D1 + k].v[p], z->v[p]);
      if (P == 1) memset(z->v[1], 0, sizeof(z->v[1]));
    }
  int st = linsolve_internal(K, P, N, n, d, as, bs, dxs, rdiag_abs, method);
  if (!st) {
    double nd = 0.0, ninf = 0.0;
    for (int k = 0; k <= d; ++k)
      for (int i = 0; i < n; ++i) {
        mdc *xi = &xs[(long)i * D1 + k];
        const mdc *di = &dxs[(long)k * n + i];
        c_add(K, P, xi, di, xi);
        double re = di->v[0][0], im = (P == 2) ? di->v[1][0] : 0.0;
        double mod = sqrt(re * re + im * im);
        if (mod > ninf) ninf = mod;
        if (k == d && mod > nd) nd = mod;
      }
    store_series(K, P, n, d, xs, x);
    if (dxnorm) {
      dxnorm[0] = nd;
      dxnorm[1] = ninf;
    }
  }
  free(coefs);
  free(csts);
  free(xs);
  free(fs);
  free(as);
  free(bs);
  free(dxs);
  return st;
}

int orc_newton_step_m(int K, int cplx, int n, int d, int nmono, const int *poly_ptr, const int *nvar, const int *idx,
                      const int *expo, const double *coef, const double *cst, double *x, double *dxnorm,
                      double *rdiag_abs, int method) {
  return orc_newton_step_ls(K, cplx, n, n, d, nmono, poly_ptr, nvar, idx, expo, coef, cst, x, dxnorm, rdiag_abs,
                            method);
}

int orc_newton_step(int K, int cplx, int n, int d, int nmono, const int *poly_ptr, const int *nvar, const int *idx,
                    const int *expo, const double *coef, const double *cst, double *x, double *dxnorm, double *rdiag_abs) {
  return orc_newton_step_m(K, cplx, n, d, nmono, poly_ptr, nvar, idx, expo, coef, cst, x, dxnorm, rdiag_abs, 0);
}

/* ------------------------------------- Newton with degree continuation */
/*
 * The driver of the cyclic 128-roots run in Sec. 6: levels l = 0..nlev-1 at
 * truncation degrees deg[l].  Level l takes Newton steps on coefficients
 * 0..deg[l] of x, at most maxit[l] of them, and ends early once ||dx|| (the
 * update of the last coefficient, dxnorm[0] above) is <= tol.  The next level
 * starts from this one's series.  The ladder stops after a level whose last
 * ||dx|| is above too_large (the paper gives no number for "too large"; the
 * caller does).  x: [P][K][n][D+1] in and out.  Per level: iters[l], the final
 * ||dx|| in dxn[2l] and max |dx| in dxn[2l+1]; *levels = levels run.
 */
int orc_newton_run(int K, int cplx, int N, int n, int D, int nmono, const int *poly_ptr, const int *nvar, const int *idx,
                   const int *expo, const double *coef, const double *cst, double *x, int nlev, const int *deg,
                   const int *maxit, double tol, double too_large, int *iters, double *dxn, int *levels, int method) {
  int P = cplx ? 2 : 1;
  if (check_system(K, N, n, D, nmono, poly_ptr, nvar, idx, expo) || nlev < 1) return 1;
  for (int l = 0; l < nlev; ++l)
    if (deg[l] < 0 || deg[l] > D || (l > 0 && deg[l] < deg[l - 1]) || maxit[l] < 1) return 1;
  long rows = (long)P * K * n;
  double *xl = malloc(sizeof(double) * rows * (D + 1));
  int st = 0;
  *levels = 0;
  for (int l = 0; l < nlev && !st; ++l) {
    int d = deg[l];
    for (long r = 0; r < rows; ++r)
      for (int k = 0; k <= d; ++k) xl[r * (d + 1) + k] = x[r * (D + 1) + k];
    double nrm[2] = {0.0, 0.0};
    int it = 0;
    while (it < maxit[l]) {
      st = orc_newton_step_ls(K, cplx, N, n, d, nmono, poly_ptr, nvar, idx, expo, coef, cst, xl, nrm, NULL, method);
      if (st) break;
      ++it;
      if (nrm[0] <= tol) break;
    }
    for (long r = 0; r < rows; ++r)
      for (int k = 0; k <= d; ++k) x[r * (D + 1) + k] = xl[r * (d + 1) + k];
    iters[l] = it;
    dxn[2 * l] = nrm[0];
    dxn[2 * l + 1] = nrm[1];
    *levels = l + 1;
    if (!(nrm[0] <= too_large)) break;
  }
  free(xl);
  return st;
}

/* --------------------------------------------------- condition of A_0 */
/*
 * 1 / (||A_0||_1 ||A_0^{-1}||_1) (Sec. 6 quotes an estimate of the inverse
 * condition number of A_0).  A_0^{-1} (the pseudo-inverse when N > n) is
 * computed column by column by solving A_0 x = e_c with the factorisation of
 * `method`; the 1-norms use the moduli of the leading limbs, summed in double
 * down each column.  A: [P][K][d+1][n][N] as for orc_lstsq (coefficient 0).
 */
int orc_rcond(int K, int cplx, int N, int n, int d, const double *A, int method, double *out) {
  int P = cplx ? 2 : 1;
  if (K < 1 || K > MAXK || n < 1 || N < n || d < 0) return 1;
  long nn = (long)N * n;
  mdc *as = malloc(sizeof(mdc) * (d + 1) * nn);
  load_mats(K, P, N, n, d, A, as);
  fact f;
  int st = fact_init(&f, method, K, P, N, n, as);
  if (!st) {
    mdc *e = malloc(sizeof(mdc) * N), *x = malloc(sizeof(mdc) * n);
    double na = 0.0, ni = 0.0;
    for (int c = 0; c < n; ++c) { /* ||A_0||_1: N rows of column c */
      double sa = 0.0;
      for (int r = 0; r < N; ++r) {
        const mdc *a = &as[(long)r * n + c];
        double re = a->v[0][0], im = P == 2 ? a->v[1][0] : 0.0;
        sa += sqrt(re * re + im * im);
      }
      if (sa > na) na = sa;
    }
    for (int c = 0; c < N; ++c) { /* column c of the (pseudo-)inverse: n rows */
      for (int i = 0; i < N; ++i) c_zero(&e[i]);
      e[c].v[0][0] = 1.0;
      fact_solve(&f, e, x);
      double si = 0.0;
      for (int r = 0; r < n; ++r) {
        double re = x[r].v[0][0], im = P == 2 ? x[r].v[1][0] : 0.0;
        si += sqrt(re * re + im * im);
      }
      if (si > ni) ni = si;
    }
    *out = 1.0 / (na * ni);
    free(e);
    free(x);
  }
  fact_free(&f);
  free(as);
  return st;
}

int orc_set_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
  return omp_get_max_threads();
#else
  (void)t;
  return 1;
#endif
}
