/*
 * Oracle for the look-ahead decentralized particle filter (LA-DPF) step.
 *
 * TEST INFRASTRUCTURE ONLY. This file is a plain, slow, FP64, single-purpose C
 * restatement of the method of "Decentralized, Adaptive, Look-Ahead Particle
 * Filtering" (Ahmed, Bibalan, de Freitas, Fauvel; arXiv:1203.2394). Only the
 * tests, the smoke check and the CPU-baseline leg of the benchmark may load it.
 * It shares no code, header, table or constant generator with the CUDA library;
 * the product path never calls it.
 *
 * Every function names the passage of the paper it follows. Where the paper is
 * silent, the reading taken is stated in the comment (the same readings are
 * listed in the design notes of the repository).
 *
 * Layout (array-of-structures, as is natural in C):
 *   x[i*d1 + c]            outer particles x^{(i)}, i < N
 *   z[(i*M + j)*d2 + c]    inner particles z^{(i,j)}, j < M
 *   lq[i*M + j]            log of the normalised inner weights qbar^{(i,j)}
 *   xbb[(i*L + m)*d1 + c]  look-ahead draws xbarbar^{(m)} of outer particle i
 *   lwhat[i*L + m]         log of the per-draw look-ahead weight
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11) with key (seed_lo, seed_hi ^ filter_id)
 * and counter (t, i, purpose<<24 | sub, block). Normals come from the
 * Box-Muller transform of two 32-bit words. The CUDA library implements the
 * same published generator independently, so both consume identical words.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORA_OK 0
#define ORA_E_INVALID 1
#define ORA_E_NOMEM 2
#define ORA_E_NUMERIC 5

/* Purposes of random draws (the counter's third word carries purpose<<24). */
enum {
  P_INIT_X = 1, P_INIT_Z = 2, P_LA_J = 3, P_LA_X = 4, P_LA_Z = 5,
  P_OUTER = 6, P_SEL = 7, P_INNER = 8, P_PROP = 9
};

static const double LOG_2PI = 1.8378770664093454835606594728112;

/* ------------------------------------------------------------------------- */
/* Philox4x32-10, from its definition in Salmon et al. (SC'11): ten rounds of  */
/* two 32x32->64 multiplications, the high halves xor-ed with the other       */
/* counter words and the round key, the key bumped by the Weyl constants.     */
/* ------------------------------------------------------------------------- */
void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

typedef struct {
  uint32_t key[2];
} ora_rng;

static ora_rng rng_make(uint64_t seed, uint32_t filter_id) {
  ora_rng r;
  r.key[0] = (uint32_t)seed;
  r.key[1] = (uint32_t)(seed >> 32) ^ filter_id;
  return r;
}

static void rng_block(const ora_rng* r, uint32_t t, uint32_t i, uint32_t purpose, uint32_t sub,
                      uint32_t block, uint32_t out[4]) {
  uint32_t ctr[4] = {t, i, (purpose << 24) | (sub & 0xFFFFFFu), block};
  ora_philox4x32_10(ctr, r->key, out);
}

/* One 32-bit word: word 0 of block 0. */
static uint32_t rng_word(const ora_rng* r, uint32_t t, uint32_t i, uint32_t purpose, uint32_t sub) {
  uint32_t w[4];
  rng_block(r, t, i, purpose, sub, 0, w);
  return w[0];
}

/* Uniform on (0,1): ((w >> 9) + 1/2) * 2^-23, exact in binary32 and binary64. */
double ora_u01(uint32_t w) { return ((double)(w >> 9) + 0.5) * 0x1p-23; }

/* Box-Muller: two words give two independent standard normals. */
void ora_box_muller(uint32_t wa, uint32_t wb, double* n0, double* n1) {
  double ua = ora_u01(wa), ub = ora_u01(wb);
  double rad = sqrt(-2.0 * log(ua));
  double th = 2.0 * M_PI * ub;
  *n0 = rad * cos(th);
  *n1 = rad * sin(th);
}

/* n standard normals for (t, i, purpose, sub): pair p uses words 2(p mod 2),
 * 2(p mod 2)+1 of block p/2. */
static void rng_normals(const ora_rng* r, uint32_t t, uint32_t i, uint32_t purpose, uint32_t sub,
                        int n, double* out) {
  uint32_t w[4];
  for (int p = 0; 2 * p < n; ++p) {
    if (p % 2 == 0) rng_block(r, t, i, purpose, sub, (uint32_t)(p / 2), w);
    double a, b;
    ora_box_muller(w[2 * (p % 2)], w[2 * (p % 2) + 1], &a, &b);
    out[2 * p] = a;
    if (2 * p + 1 < n) out[2 * p + 1] = b;
  }
}

/* The dy normals of the look-ahead's common inner draw of inner particle k (purpose
 * LA_Z). For dy <= 2 two inner particles share one Philox block: particle k takes the
 * Box-Muller pair of words 2(k mod 2), 2(k mod 2)+1 of block (t, i, LA_Z, k / 2) (dy = 1
 * keeps its first normal); for dy > 2 they are the normals of (t, i, LA_Z, k). */
static void rng_la_z(const ora_rng* r, uint32_t t, uint32_t i, uint32_t k, int dy, double* out) {
  if (dy <= 2) {
    uint32_t w[4];
    rng_block(r, t, i, P_LA_Z, k >> 1, 0, w);
    double a, b;
    ora_box_muller(w[2 * (k & 1)], w[2 * (k & 1) + 1], &a, &b);
    out[0] = a;
    if (dy > 1) out[1] = b;
  } else {
    rng_normals(r, t, i, P_LA_Z, k, dy, out);
  }
}

/* Exposed for the generator tests. */
void ora_normals(uint64_t seed, uint32_t filter_id, uint32_t t, uint32_t i, uint32_t purpose,
                 uint32_t sub, int n, double* out) {
  ora_rng r = rng_make(seed, filter_id);
  rng_normals(&r, t, i, purpose, sub, n, out);
}

/* Many keys at once: row q of out (n values) holds the normals of
 * (t, idx[q], purpose, sub[q]); for the oracles written in numpy. */
void ora_normals_many(uint64_t seed, uint32_t filter_id, uint32_t t, int64_t count,
                      const uint32_t* idx, uint32_t purpose, const uint32_t* sub, int n,
                      double* out) {
  ora_rng r = rng_make(seed, filter_id);
  for (int64_t q = 0; q < count; ++q) rng_normals(&r, t, idx[q], purpose, sub[q], n, out + q * n);
}

/* ------------------------------------------------------------------------- */
/* Systematic resampling ("standard resampling", steps 2 and 6 of the DPF,    */
/* step 3 of the LA-DPF). The paper does not name the scheme; the systematic  */
/* scheme is taken, in an exact integer form:                                 */
/*   e   = floor(log2(max W)),  B = ceil(log2 n)                              */
/*   c_i = floor(W_i * 2^(S - e))          (an exact scaling, then a floor)    */
/*   cum_i = c_0 + ... + c_i,  C = cum_{n-1}                                  */
/*   a_k = min{ i : cum_i * n_out * 2^b > (k * 2^b + u_b) * C }                */
/* i.e. the first i whose cumulative weight exceeds the k-th systematic point */
/* (k + U) C / n_out with U = u_b / 2^b.                                      */
/* Global rule: S = 62 - B, b = 32, 128-bit products (any n < 2^31).          */
/* Local rule:  S = 31 - B, b = 16 (b = 32 when n_out = 1), 64-bit products,  */
/*              n <= 1024.                                                    */
/* ------------------------------------------------------------------------- */
static int ceil_log2(int64_t n) {
  int b = 0;
  while (((int64_t)1 << b) < n) ++b;
  return b;
}

/* Returns 0 and fills c, or ORA_E_NUMERIC when no weight is positive. */
static int quantize(const double* W, int64_t n, int S, uint64_t* c) {
  double wmax = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    if (!(W[i] >= 0.0) || isinf(W[i])) return ORA_E_NUMERIC;
    if (W[i] > wmax) wmax = W[i];
  }
  if (wmax == 0.0) return ORA_E_NUMERIC;
  int e = ilogb(wmax);
  for (int64_t i = 0; i < n; ++i) c[i] = (uint64_t)floor(ldexp(W[i], S - e));
  return ORA_OK;
}

int ora_sys_global(const double* W, int64_t n, uint32_t u, int32_t* out) {
  if (n <= 0) return n == 0 ? ORA_OK : ORA_E_INVALID;
  if (n >= ((int64_t)1 << 31)) return ORA_E_INVALID;
  uint64_t* c = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)n);
  if (!c) return ORA_E_NOMEM;
  int st = quantize(W, n, 62 - ceil_log2(n), c);
  if (st) { free(c); return st; }
  for (int64_t i = 1; i < n; ++i) c[i] += c[i - 1]; /* now the inclusive cumulative sum */
  unsigned __int128 C = c[n - 1];
  int64_t i = 0;
  for (int64_t k = 0; k < n; ++k) {
    unsigned __int128 rhs = (((unsigned __int128)k << 32) + u) * C;
    while ((unsigned __int128)c[i] * (unsigned __int128)n * ((unsigned __int128)1 << 32) <= rhs) ++i;
    out[k] = (int32_t)i;
  }
  free(c);
  return ORA_OK;
}

int ora_sys_local(const double* W, int n, int n_out, uint32_t u, int32_t* out) {
  if (n <= 0 || n > 1024 || n_out <= 0 || n_out > 1024) return ORA_E_INVALID;
  uint64_t c[1024];
  int st = quantize(W, n, 31 - ceil_log2(n), c);
  if (st) return st;
  for (int i = 1; i < n; ++i) c[i] += c[i - 1];
  uint64_t C = c[n - 1];
  int b = (n_out == 1) ? 32 : 16;
  uint64_t ub = (n_out == 1) ? (uint64_t)u : (uint64_t)(u >> 16);
  int i = 0;
  for (int k = 0; k < n_out; ++k) {
    uint64_t rhs = (((uint64_t)k << b) + ub) * C;
    while (c[i] * (uint64_t)n_out * ((uint64_t)1 << b) <= rhs) ++i;
    out[k] = i;
  }
  return ORA_OK;
}

/* ------------------------------------------------------------------------- */
/* Small dense linear algebra (row-major).                                    */
/* ------------------------------------------------------------------------- */
/* Lower Cholesky factor of an SPD matrix; returns 0 on success. */
static int chol(const double* S, int n, double* Lo) {
  memset(Lo, 0, sizeof(double) * (size_t)(n * n));
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j <= i; ++j) {
      double s = S[i * n + j];
      for (int k = 0; k < j; ++k) s -= Lo[i * n + k] * Lo[j * n + k];
      if (i == j) {
        if (!(s > 0.0)) return 1;
        Lo[i * n + i] = sqrt(s);
      } else {
        Lo[i * n + j] = s / Lo[j * n + j];
      }
    }
  }
  return 0;
}

/* Solve Lo v = b (forward substitution). */
static void fwd_solve(const double* Lo, int n, const double* b, double* v) {
  for (int i = 0; i < n; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= Lo[i * n + k] * v[k];
    v[i] = s / Lo[i * n + i];
  }
}

/* log N(v; 0, Lo Lo^T) with its full normalising constant. */
static double log_normal(const double* Lo, int n, const double* v) {
  double w[64];
  fwd_solve(Lo, n, v, w);
  double q = 0.0, ld = 0.0;
  for (int i = 0; i < n; ++i) {
    q += w[i] * w[i];
    ld += log(Lo[i * n + i]);
  }
  return -0.5 * q - ld - 0.5 * n * LOG_2PI;
}

/* out = Lo * e (lower triangular times vector) */
static void tri_mul(const double* Lo, int n, const double* e, double* out) {
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int k = 0; k <= i; ++k) s += Lo[i * n + k] * e[k];
    out[i] = s;
  }
}

/* Invert an SPD matrix through its Cholesky factor (columns by solves). */
static int spd_inverse(const double* S, int n, double* Sinv) {
  double Lo[64 * 64], e[64], v[64], w[64];
  if (chol(S, n, Lo)) return 1;
  for (int c = 0; c < n; ++c) {
    for (int i = 0; i < n; ++i) e[i] = (i == c) ? 1.0 : 0.0;
    fwd_solve(Lo, n, e, v);
    /* back substitution with Lo^T */
    for (int i = n - 1; i >= 0; --i) {
      double s = v[i];
      for (int k = i + 1; k < n; ++k) s -= Lo[k * n + i] * w[k];
      w[i] = s / Lo[i * n + i];
    }
    for (int i = 0; i < n; ++i) Sinv[i * n + c] = w[i];
  }
  return 0;
}

/* log-sum-exp of n values (the plain max-shifted definition). */
static double lse(const double* v, int64_t n) {
  double mx = -INFINITY;
  for (int64_t i = 0; i < n; ++i) if (v[i] > mx) mx = v[i];
  if (mx == -INFINITY) return -INFINITY;
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += exp(v[i] - mx);
  return mx + log(s);
}

/* ------------------------------------------------------------------------- */
/* The state-space model (eq. mainDPF):                                        */
/*   x_{t+1} = f^x(x_t, z_t, t) + v^x,   v^x ~ N(0, Q_x)                        */
/*   z_{t+1} = f^z(x_t, z_t)    + v^z,   v^z ~ N(0, Q_z)                        */
/*   y_t     = h(x_t, z_t)      + e_t,   e_t ~ N(0, R)                          */
/* in the conditionally linear-Gaussian family                                 */
/*   f^x = g(x, t) + A_xx x + A_xz z,  g = a x + b x/(1+x^2) + c cos(w t)       */
/*         per coordinate when enabled (the growth map of Table 1);            */
/*   f^z = A_zx x + A_zz z;                                                    */
/*   h   = q x.^2 + H_x x + H_z z  (the x.^2 term when enabled, dy = d1).      */
/* The process noise is independent between the blocks (Q block-diagonal), so */
/* p(z_{t+1} | x_{t:t+1}, z_t) does not depend on x_{t+1}.                      */
/* Initial law: [x_0; z_0] ~ N(m0, P0).                                        */
/* ------------------------------------------------------------------------- */
typedef struct {
  int32_t d1, d2, dy;
  int32_t growth_x;
  int32_t quad_obs;
  int32_t reserved;
  double ga, gb, gc, gw, qc;
  const double* A;  /* d x d */
  const double* Q;  /* d x d, zero off-diagonal blocks */
  const double* H;  /* dy x d */
  const double* R;  /* dy x dy */
  const double* m0; /* d */
  const double* P0; /* d x d */
} ora_model_in;

typedef struct {
  int d1, d2, dy, d;
  int growth_x, quad_obs;
  double ga, gb, gc, gw, qc;
  double Axx[64 * 64], Axz[64 * 64], Azx[64 * 64], Azz[64 * 64];
  double Hx[64 * 64], Hz[64 * 64];
  double Lqx[64 * 64], Lqz[64 * 64], Lr[64 * 64];
  double Ls[64 * 64];     /* Cholesky of S = H_z Q_z H_z^T */
  double K[64 * 64];      /* Q_z H_z^T S^{-1} (d2 x dy) */
  double m0x[64], m0z[64];
  double Lp0x[64 * 64];   /* Cholesky of P0_xx */
  double G0[64 * 64];     /* P0_zx P0_xx^{-1} (d2 x d1) */
  double Lp0c[64 * 64];   /* Cholesky of P0_zz - G0 P0_xz */
} ora_model;

static int model_prepare(const ora_model_in* in, ora_model* m) {
  int d1 = in->d1, d2 = in->d2, dy = in->dy, d = d1 + d2;
  if (d1 < 1 || d2 < 1 || dy < 1 || d1 > 64 || d2 > 64 || dy > 64) return ORA_E_INVALID;
  if (in->quad_obs && dy != d1) return ORA_E_INVALID;
  memset(m, 0, sizeof(*m));
  m->d1 = d1; m->d2 = d2; m->dy = dy; m->d = d;
  m->growth_x = in->growth_x; m->quad_obs = in->quad_obs;
  m->ga = in->ga; m->gb = in->gb; m->gc = in->gc; m->gw = in->gw; m->qc = in->qc;
  for (int r = 0; r < d1; ++r) {
    for (int c = 0; c < d1; ++c) m->Axx[r * d1 + c] = in->A[r * d + c];
    for (int c = 0; c < d2; ++c) m->Axz[r * d2 + c] = in->A[r * d + d1 + c];
  }
  for (int r = 0; r < d2; ++r) {
    for (int c = 0; c < d1; ++c) m->Azx[r * d1 + c] = in->A[(d1 + r) * d + c];
    for (int c = 0; c < d2; ++c) m->Azz[r * d2 + c] = in->A[(d1 + r) * d + d1 + c];
  }
  for (int r = 0; r < dy; ++r) {
    for (int c = 0; c < d1; ++c) m->Hx[r * d1 + c] = in->H[r * d + c];
    for (int c = 0; c < d2; ++c) m->Hz[r * d2 + c] = in->H[r * d + d1 + c];
  }
  double Qx[64 * 64], Qz[64 * 64];
  for (int r = 0; r < d; ++r)
    for (int c = 0; c < d; ++c) {
      double q = in->Q[r * d + c];
      int rx = r < d1, cx = c < d1;
      if (rx != cx && q != 0.0) return ORA_E_INVALID; /* cross-block noise not in this family */
      if (rx && cx) Qx[r * d1 + c] = q;
      if (!rx && !cx) Qz[(r - d1) * d2 + (c - d1)] = q;
    }
  if (chol(Qx, d1, m->Lqx) || chol(Qz, d2, m->Lqz) || chol(in->R, dy, m->Lr)) return ORA_E_INVALID;
  /* S = H_z Q_z H_z^T and the gain K = Q_z H_z^T S^{-1} */
  double S[64 * 64], QHt[64 * 64], Sinv[64 * 64];
  for (int r = 0; r < d2; ++r)
    for (int c = 0; c < dy; ++c) {
      double s = 0.0;
      for (int k = 0; k < d2; ++k) s += Qz[r * d2 + k] * m->Hz[c * d2 + k];
      QHt[r * dy + c] = s;
    }
  for (int r = 0; r < dy; ++r)
    for (int c = 0; c < dy; ++c) {
      double s = 0.0;
      for (int k = 0; k < d2; ++k) s += m->Hz[r * d2 + k] * QHt[k * dy + c];
      S[r * dy + c] = s;
    }
  if (chol(S, dy, m->Ls) || spd_inverse(S, dy, Sinv)) return ORA_E_INVALID;
  for (int r = 0; r < d2; ++r)
    for (int c = 0; c < dy; ++c) {
      double s = 0.0;
      for (int k = 0; k < dy; ++k) s += QHt[r * dy + k] * Sinv[k * dy + c];
      m->K[r * dy + c] = s;
    }
  /* initial law: x0 ~ N(m0x, P0xx); z0 | x0 ~ N(m0z + G0 (x0 - m0x), P0zz - G0 P0xz) */
  double Pxx[64 * 64], Pxxinv[64 * 64], Pc[64 * 64];
  for (int r = 0; r < d1; ++r) {
    m->m0x[r] = in->m0[r];
    for (int c = 0; c < d1; ++c) Pxx[r * d1 + c] = in->P0[r * d + c];
  }
  for (int r = 0; r < d2; ++r) m->m0z[r] = in->m0[d1 + r];
  if (chol(Pxx, d1, m->Lp0x) || spd_inverse(Pxx, d1, Pxxinv)) return ORA_E_INVALID;
  for (int r = 0; r < d2; ++r)
    for (int c = 0; c < d1; ++c) {
      double s = 0.0;
      for (int k = 0; k < d1; ++k) s += in->P0[(d1 + r) * d + k] * Pxxinv[k * d1 + c];
      m->G0[r * d1 + c] = s;
    }
  for (int r = 0; r < d2; ++r)
    for (int c = 0; c < d2; ++c) {
      double s = in->P0[(d1 + r) * d + d1 + c];
      for (int k = 0; k < d1; ++k) s -= m->G0[r * d1 + k] * in->P0[k * d + d1 + c];
      Pc[r * d2 + c] = s;
    }
  if (chol(Pc, d2, m->Lp0c)) return ORA_E_INVALID;
  return ORA_OK;
}

/* f^x(x, z, s): mean of x_{s+1} given (x_s, z_s) = (x, z). */
static void f_x(const ora_model* m, const double* x, const double* z, double s, double* out) {
  for (int r = 0; r < m->d1; ++r) {
    double v = 0.0;
    if (m->growth_x)
#ifdef PLANT_GROWTH_SIGN /* planted mistake: the sign of the cosine term */
      v = m->ga * x[r] + m->gb * x[r] / (1.0 + x[r] * x[r]) - m->gc * cos(m->gw * s);
#else
      v = m->ga * x[r] + m->gb * x[r] / (1.0 + x[r] * x[r]) + m->gc * cos(m->gw * s);
#endif
    for (int c = 0; c < m->d1; ++c) v += m->Axx[r * m->d1 + c] * x[c];
    for (int c = 0; c < m->d2; ++c) v += m->Axz[r * m->d2 + c] * z[c];
    out[r] = v;
  }
}

/* f^z(x, z): mean of z_{s+1} given (x_s, z_s). */
static void f_z(const ora_model* m, const double* x, const double* z, double* out) {
  for (int r = 0; r < m->d2; ++r) {
    double v = 0.0;
    for (int c = 0; c < m->d1; ++c) v += m->Azx[r * m->d1 + c] * x[c];
#ifdef PLANT_AZZ_T /* planted mistake for the pin tests: A_zz transposed */
    for (int c = 0; c < m->d2; ++c) v += m->Azz[c * m->d2 + r] * z[c];
#else
    for (int c = 0; c < m->d2; ++c) v += m->Azz[r * m->d2 + c] * z[c];
#endif
    out[r] = v;
  }
}

/* The x-only part of the observation mean: q x.^2 + H_x x. */
static void h_x(const ora_model* m, const double* x, double* out) {
  for (int r = 0; r < m->dy; ++r) {
    double v = m->quad_obs ? m->qc * x[r] * x[r] : 0.0;
    for (int c = 0; c < m->d1; ++c) v += m->Hx[r * m->d1 + c] * x[c];
    out[r] = v;
  }
}

/* log p(x' | x, z) at source step s */
static double log_px(const ora_model* m, const double* xn, const double* x, const double* z, double s) {
  double mu[64], v[64];
  f_x(m, x, z, s, mu);
  for (int r = 0; r < m->d1; ++r) v[r] = xn[r] - mu[r];
  return log_normal(m->Lqx, m->d1, v);
}

/* log p(y | x, z) */
static double log_py(const ora_model* m, const double* y, const double* x, const double* z) {
  double hx[64], v[64];
  h_x(m, x, hx);
  for (int r = 0; r < m->dy; ++r) {
    double s = hx[r];
    for (int c = 0; c < m->d2; ++c) s += m->Hz[r * m->d2 + c] * z[c];
    v[r] = y[r] - s;
  }
  return log_normal(m->Lr, m->dy, v);
}

/* ------------------------------------------------------------------------- */
/* Filter entry points.                                                      */
/* ------------------------------------------------------------------------- */
typedef struct {
  int64_t N;
  int32_t M, L;
  uint64_t seed;
  uint32_t filter_id;
  int32_t nthreads;
} ora_dims;

static int dims_ok(const ora_dims* D) {
  return D->N >= 1 && D->N < ((int64_t)1 << 31) && D->M >= 1 && D->M <= 1024 && D->L >= 1 &&
         D->L <= 64;
}

static void set_threads(const ora_dims* D) {
#ifdef _OPENMP
  if (D->nthreads > 0) omp_set_num_threads(D->nthreads);
#else
  (void)D;
#endif
}

/* Initialisation (Fig. 4, "Initialize"): x_0^(i) ~ p(x_0), z_0^(i,j) ~ p(z_0 | x_0^(i)),
 * equal inner weights lq = -log M. There is no y_0. */
int ora_init(const ora_model_in* min, const ora_dims* D, double* x, double* z, double* lq) {
  ora_model m;
  if (!dims_ok(D)) return ORA_E_INVALID;
  int st = model_prepare(min, &m);
  if (st) return st;
  ora_rng r = rng_make(D->seed, D->filter_id);
  int d1 = m.d1, d2 = m.d2, M = D->M;
  set_threads(D);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < D->N; ++i) {
    double e[64], v[64];
    rng_normals(&r, 0, (uint32_t)i, P_INIT_X, 0, d1, e);
    tri_mul(m.Lp0x, d1, e, v);
    for (int c = 0; c < d1; ++c) x[i * d1 + c] = m.m0x[c] + v[c];
    for (int j = 0; j < M; ++j) {
      rng_normals(&r, 0, (uint32_t)i, P_INIT_Z, (uint32_t)j, d2, e);
      tri_mul(m.Lp0c, d2, e, v);
      for (int c = 0; c < d2; ++c) {
        double s = m.m0z[c] + v[c];
        for (int k = 0; k < d1; ++k) s += m.G0[c * d1 + k] * (x[i * d1 + k] - m.m0x[k]);
        z[(i * M + j) * d2 + c] = s;
      }
      lq[i * M + j] = -log((double)M);
    }
  }
  return ORA_OK;
}

/*
 * Look-ahead of one outer particle i at step t (Fig. 4 steps 1-2).
 *
 * Step 1 (eq. approx1): L draws xbb^(m) from p_Nz(x_t | x_{0:t-1}^(i)) =
 *   sum_j qbar^(i,j) p(x_t | x_{t-1}^(i), z^(i,j)): a component j_m ~ qbar (key
 *   (t,i,m,LA_J)), then xbb = f^x(x, z^(i,j_m), t-1) + chol(Q_x) eps (key (t,i,m,LA_X)).
 *   The corresponding inner draws zbb^(m,k) ~ p(z_t | x^(i)_{0:t-1}, xbb^(m), y_{0:t-1})
 *   are taken in weighted form (reading): one propagated draw per inner particle k,
 *   shared by all m, weighted for draw m by
 *     alpha^(m,k) = lq^(i,k) + log p(xbb^(m) | x^(i), z^(i,k))     (eq. qnobar, r = 1).
 *   Because the observation is linear in z, the draw enters p(y | .) only through
 *   H_z zbb; that projection is drawn directly:
 *     g^(k) = H_z f^z(x^(i), z^(i,k)) + chol(H_z Q_z H_z^T) eps   (key (t,i,k,LA_Z)),
 *   which has the law of H_z zbb^(k).
 * Step 2 (eq. weightsMC, self-normalised over the weighted inner draws):
 *   ell^(m,k)  = log p(y_t | xbb^(m), zbb^(k))
 *   lwhat^(m)  = LSE_k(alpha + ell) - LSE_k(alpha)
 *   lw         = LSE_m(lwhat) - log L     (the average over the L draws)
 * Also returns, for the filtered-mean estimate, the z-mean of each draw
 *   mu^(m) = sum_k softmax_k(alpha + ell) E[zbb^(k) | g^(k)],
 *   E[zbb | g] = f^z + K (g - H_z f^z),  K = Q_z H_z^T (H_z Q_z H_z^T)^{-1}.
 * jla (L), xbb (L*d1), lwhat (L), mu (L*d2) are outputs; lw is returned.
 */
static double lookahead_group(const ora_model* m, const ora_dims* D, const ora_rng* r, uint32_t t,
                              int64_t i, const double* x_i, const double* z_i, const double* lq_i,
                              const double* y, int32_t* jla, double* xbb, double* lwhat,
                              double* mu) {
  int d1 = m->d1, d2 = m->d2, dy = m->dy, M = D->M, L = D->L;
  double s = (double)t - 1.0; /* the source step index of the transition x_{t-1} -> x_t */
  double* W = (double*)malloc(sizeof(double) * (size_t)M);
  double* g = (double*)malloc(sizeof(double) * (size_t)(M * dy));
  double* zm = (double*)malloc(sizeof(double) * (size_t)(M * d2)); /* E[zbb^(k) | g^(k)] */
  double* a = (double*)malloc(sizeof(double) * (size_t)M);
  double* al = (double*)malloc(sizeof(double) * (size_t)M);
  double lqmax = -INFINITY;
  for (int k = 0; k < M; ++k) if (lq_i[k] > lqmax) lqmax = lq_i[k];
  for (int k = 0; k < M; ++k) W[k] = exp(lq_i[k] - lqmax);
  /* step 1: the x draws */
  for (int mm = 0; mm < L; ++mm) {
    int32_t j;
    ora_sys_local(W, M, 1, rng_word(r, t, (uint32_t)i, P_LA_J, (uint32_t)mm), &j);
    jla[mm] = j;
    double mu_x[64], e[64], v[64];
    f_x(m, x_i, z_i + (size_t)j * d2, s, mu_x);
    rng_normals(r, t, (uint32_t)i, P_LA_X, (uint32_t)mm, d1, e);
    tri_mul(m->Lqx, d1, e, v);
    for (int c = 0; c < d1; ++c) xbb[mm * d1 + c] = mu_x[c] + v[c];
  }
  /* step 1: the inner draws, projected through H_z */
  for (int k = 0; k < M; ++k) {
    double fz[64], e[64], v[64];
    f_z(m, x_i, z_i + (size_t)k * d2, fz);
    rng_la_z(r, t, (uint32_t)i, (uint32_t)k, dy, e);
    tri_mul(m->Ls, dy, e, v);
    for (int q = 0; q < dy; ++q) {
      double hz = 0.0;
      for (int c = 0; c < d2; ++c) hz += m->Hz[q * d2 + c] * fz[c];
#ifdef PLANT_NO_PROJ_NOISE /* planted mistake: the inner look-ahead draw without noise */
      g[k * dy + q] = hz;
#else
      g[k * dy + q] = hz + v[q];
#endif
    }
    for (int c = 0; c < d2; ++c) {
      double s2 = fz[c];
#ifndef PLANT_MEAN_NO_GAIN /* planted mistake: E[zbb | g] replaced by f^z */
      for (int q = 0; q < dy; ++q) s2 += m->K[c * dy + q] * v[q];
#endif
      zm[k * d2 + c] = s2;
    }
  }
  /* step 2: the weights */
  double* lwh = (double*)malloc(sizeof(double) * (size_t)L);
  for (int mm = 0; mm < L; ++mm) {
    const double* xb = xbb + mm * d1;
    double hx[64];
    h_x(m, xb, hx);
    for (int k = 0; k < M; ++k) {
#ifdef PLANT_NO_QNOBAR /* planted mistake: the p(x_t | x, z) factor of eq. qnobar dropped */
      a[k] = lq_i[k];
#else
      a[k] = lq_i[k] + log_px(m, xb, x_i, z_i + (size_t)k * d2, s);
#endif
      double v[64];
      for (int q = 0; q < dy; ++q) v[q] = y[q] - hx[q] - g[k * dy + q];
      al[k] = a[k] + log_normal(m->Lr, dy, v);
    }
    double lse_al = lse(al, M);
    lwh[mm] = lse_al - lse(a, M);
    lwhat[mm] = lwh[mm];
    for (int c = 0; c < d2; ++c) mu[mm * d2 + c] = 0.0;
    if (lse_al > -INFINITY)
      for (int k = 0; k < M; ++k) {
        double wk = exp(al[k] - lse_al);
        for (int c = 0; c < d2; ++c) mu[mm * d2 + c] += wk * zm[k * d2 + c];
      }
  }
#ifdef PLANT_NO_AVERAGE /* planted mistake: the 1/L of eq. weightsMC dropped */
  double lw = lse(lwh, L);
#else
  double lw = lse(lwh, L) - log((double)L);
#endif
  free(lwh); free(W); free(g); free(zm); free(a); free(al);
  return lw;
}

/*
 * Step 4 of Fig. 4 for one destination i ("generate new particles"), given its
 * ancestor a (the outer resampling of step 3) and its new x_t^(i):
 *   local resampling (DPF step 6) of the ancestor's inner set by
 *     alpha^(k) = lq^(a,k) + log p(x_t^(i) | x^(a), z^(a,k))   (eq. qnobar, r = 1),
 *     systematic, key (t,i,0,INNER);
 *   propagation z_t^(i,j) = f^z(x^(a), z^(a,b_j)) + chol(Q_z) eps, key (t,i,j,PROP)
 *     (the prior proposal p(z_t | x_{0:t}, y_{0:t-1}) of section 2.1, so r = 1);
 *   measurement update (eq. qbar): lq_t^(i,j) = ell_j - LSE_j ell,
 *     ell_j = log p(y_t | x_t^(i), z_t^(i,j)).
 * bidx_in (optional): replay the given local resampling indices instead of drawing
 * them (the rest of the step is unchanged); alpha_out (optional): the M weights alpha.
 */
static int finalize_group(const ora_model* m, const ora_dims* D, const ora_rng* r, uint32_t t,
                          int64_t i, const double* xa, const double* za, const double* lqa,
                          const double* xn, const double* y, double* zn, double* lqn,
                          int32_t* bidx, const int32_t* bidx_in, double* alpha_out) {
  int d2 = m->d2, M = D->M;
  double s = (double)t - 1.0;
  double* al = (double*)malloc(sizeof(double) * (size_t)M);
  double* W = (double*)malloc(sizeof(double) * (size_t)M);
#ifdef PLANT_NO_QNOBAR
  for (int k = 0; k < M; ++k) al[k] = lqa[k];
#else
  for (int k = 0; k < M; ++k) al[k] = lqa[k] + log_px(m, xn, xa, za + (size_t)k * d2, s);
#endif
  double mx = -INFINITY;
  for (int k = 0; k < M; ++k) if (al[k] > mx) mx = al[k];
  for (int k = 0; k < M; ++k) W[k] = exp(al[k] - mx);
  if (alpha_out)
    for (int k = 0; k < M; ++k) alpha_out[k] = al[k];
  int st = ORA_OK;
  if (bidx_in) { /* replay: the local resampling indices are given */
    for (int j = 0; j < M; ++j) {
      if (bidx_in[j] < 0 || bidx_in[j] >= M) { free(al); free(W); return ORA_E_INVALID; }
      bidx[j] = bidx_in[j];
    }
  } else {
    st = ora_sys_local(W, M, M, rng_word(r, t, (uint32_t)i, P_INNER, 0), bidx);
  }
  if (st) { free(al); free(W); return st; }
  for (int j = 0; j < M; ++j) {
    double fz[64], e[64], v[64];
    f_z(m, xa, za + (size_t)bidx[j] * d2, fz);
    rng_normals(r, t, (uint32_t)i, P_PROP, (uint32_t)j, d2, e);
    tri_mul(m->Lqz, d2, e, v);
    for (int c = 0; c < d2; ++c) zn[j * d2 + c] = fz[c] + v[c];
    al[j] = log_py(m, y, xn, zn + (size_t)j * d2);
  }
  double l = lse(al, M);
  for (int j = 0; j < M; ++j) lqn[j] = al[j] - l;
  free(al); free(W);
  return ORA_OK;
}

/* Look-ahead of the given outer particles only (for sampled comparisons at large N). */
int ora_lookahead(const ora_model_in* min, const ora_dims* D, uint32_t t, const double* y,
                  int64_t n_idx, const int64_t* idx, const double* x, const double* z,
                  const double* lq, double* lw, int32_t* jla, double* xbb, double* lwhat,
                  double* mu) {
  ora_model m;
  if (!dims_ok(D) || t < 1) return ORA_E_INVALID;
  int st = model_prepare(min, &m);
  if (st) return st;
  ora_rng r = rng_make(D->seed, D->filter_id);
  int d1 = m.d1, d2 = m.d2, M = D->M, L = D->L;
  set_threads(D);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t q = 0; q < n_idx; ++q) {
    int64_t i = idx[q];
    lw[q] = lookahead_group(&m, D, &r, t, i, x + i * d1, z + i * M * d2, lq + i * M, y,
                            jla + q * L, xbb + q * L * d1, lwhat + q * L, mu + q * L * d2);
  }
  return ORA_OK;
}

/* Step 4 for the given destinations only (for sampled comparisons at large N).
 * bidx_in and alpha_out may be NULL (see finalize_group). */
int ora_finalize(const ora_model_in* min, const ora_dims* D, uint32_t t, const double* y,
                 int64_t n_idx, const int64_t* idx, const int32_t* anc, const double* x_prev,
                 const double* z_prev, const double* lq_prev, const double* x_new, double* z_new,
                 double* lq_new, int32_t* bidx, const int32_t* bidx_in, double* alpha_out) {
  ora_model m;
  if (!dims_ok(D) || t < 1) return ORA_E_INVALID;
  int st = model_prepare(min, &m);
  if (st) return st;
  ora_rng r = rng_make(D->seed, D->filter_id);
  int d1 = m.d1, d2 = m.d2, M = D->M;
  int bad = 0;
  set_threads(D);
#pragma omp parallel for schedule(dynamic, 16) reduction(| : bad)
  for (int64_t q = 0; q < n_idx; ++q) {
    int64_t i = idx[q];
    int64_t a = anc[q];
    bad |= finalize_group(&m, D, &r, t, i, x_prev + a * d1, z_prev + a * M * d2, lq_prev + a * M,
                          x_new + q * d1, y, z_new + q * M * d2, lq_new + q * M, bidx + q * M,
                          bidx_in ? bidx_in + q * M : NULL, alpha_out ? alpha_out + q * M : NULL);
  }
  return bad ? ORA_E_NUMERIC : ORA_OK;
}

/*
 * One full LA-DPF step t >= 1 (Fig. 4, in its order), from the state at t-1
 * (x_prev, z_prev, lq_prev) to the state at t (x_new, z_new, lq_new).
 *   1-2. look-ahead and weights for every outer particle (lookahead_group);
 *        logZ_t = LSE_i(lw) - log N estimates log p(y_t | y_{1:t-1}) (eq. weightsopt).
 *   3.   outer resampling: a = systematic-global(exp(lw - max), key (t,0,0,OUTER)).
 *   4.   x_t^(i) ~ pi-hat (eq. approx3) by sampling-importance-resampling over the
 *        ancestor's L look-ahead draws: m_i = systematic-local, one draw, of
 *        exp(lwhat^(a_i,.) - max), key (t,i,0,SEL); x_t^(i) = xbb^(a_i, m_i);
 *        then the inner step of finalize_group.
 * The filtered mean is the importance-weighted look-ahead estimate taken before
 * resampling: sum over (i,m) of W^(i,m) [xbb^(i,m); mu^(i,m)], W proportional
 * to exp(lwhat). mean has d1 + d2 entries (x block first).
 * Replay (anc_in, sel_in, bidx_in; each may be NULL): the outer ancestors, the
 * selected draws and the local resampling indices are taken as given instead of
 * drawn, every other quantity computed as above.
 */
int ora_step(const ora_model_in* min, const ora_dims* D, uint32_t t, const double* y,
             const double* x_prev, const double* z_prev, const double* lq_prev, double* x_new,
             double* z_new, double* lq_new, double* lw, double* lwhat, double* xbb, int32_t* jla,
             int32_t* anc, int32_t* sel, int32_t* bidx, double* mean, double* logZ,
             double* ess, const int32_t* anc_in, const int32_t* sel_in, const int32_t* bidx_in) {
  ora_model m;
  if (!dims_ok(D) || t < 1) return ORA_E_INVALID;
  int st = model_prepare(min, &m);
  if (st) return st;
  ora_rng r = rng_make(D->seed, D->filter_id);
  int64_t N = D->N;
  int d1 = m.d1, d2 = m.d2, M = D->M, L = D->L;
  double* mu = (double*)malloc(sizeof(double) * (size_t)(N * L * d2));
  if (!mu) return ORA_E_NOMEM;
  set_threads(D);
  /* steps 1-2 */
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < N; ++i)
    lw[i] = lookahead_group(&m, D, &r, t, i, x_prev + i * d1, z_prev + i * M * d2, lq_prev + i * M,
                            y, jla + i * L, xbb + i * L * d1, lwhat + i * L, mu + i * L * d2);
  double lwmax = -INFINITY;
  for (int64_t i = 0; i < N; ++i) if (lw[i] > lwmax) lwmax = lw[i];
  if (!(lwmax > -INFINITY) || isnan(lwmax)) { free(mu); return ORA_E_NUMERIC; }
  *logZ = lse(lw, N) - log((double)N);
  double s1 = 0.0, s2 = 0.0;
  for (int64_t i = 0; i < N; ++i) {
    double w = exp(lw[i] - lwmax);
    s1 += w;
    s2 += w * w;
  }
  *ess = s1 * s1 / s2;
  /* filtered mean (weights over all (i, m) pairs) */
  double lwhmax = -INFINITY;
  for (int64_t q = 0; q < N * L; ++q) if (lwhat[q] > lwhmax) lwhmax = lwhat[q];
  double sw = 0.0;
  for (int c = 0; c < d1 + d2; ++c) mean[c] = 0.0;
  for (int64_t q = 0; q < N * L; ++q) {
    double w = exp(lwhat[q] - lwhmax);
    sw += w;
    for (int c = 0; c < d1; ++c) mean[c] += w * xbb[q * d1 + c];
    for (int c = 0; c < d2; ++c) mean[d1 + c] += w * mu[q * d2 + c];
  }
  for (int c = 0; c < d1 + d2; ++c) mean[c] /= sw;
  free(mu);
  /* step 3 */
  double* W = (double*)malloc(sizeof(double) * (size_t)N);
  if (!W) return ORA_E_NOMEM;
  for (int64_t i = 0; i < N; ++i) W[i] = exp(lw[i] - lwmax);
  if (anc_in) {
    for (int64_t i = 0; i < N; ++i) {
      if (anc_in[i] < 0 || anc_in[i] >= N) { free(W); return ORA_E_INVALID; }
      anc[i] = anc_in[i];
    }
  } else {
    st = ora_sys_global(W, N, rng_word(&r, t, 0, P_OUTER, 0), anc);
  }
  free(W);
  if (st) return st;
  /* step 4 */
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : bad)
  for (int64_t i = 0; i < N; ++i) {
    int64_t a = anc[i];
    double Wm[64], mx = -INFINITY;
    for (int mm = 0; mm < L; ++mm) if (lwhat[a * L + mm] > mx) mx = lwhat[a * L + mm];
    for (int mm = 0; mm < L; ++mm) Wm[mm] = exp(lwhat[a * L + mm] - mx);
    int32_t mi = 0;
    if (sel_in) {
      mi = sel_in[i];
      if (mi < 0 || mi >= L) { bad |= ORA_E_INVALID; mi = 0; }
    } else {
      bad |= ora_sys_local(Wm, L, 1, rng_word(&r, t, (uint32_t)i, P_SEL, 0), &mi);
    }
    sel[i] = mi;
    for (int c = 0; c < d1; ++c) x_new[i * d1 + c] = xbb[(a * L + mi) * d1 + c];
    bad |= finalize_group(&m, D, &r, t, i, x_prev + a * d1, z_prev + a * M * d2, lq_prev + a * M,
                          x_new + i * d1, y, z_new + i * M * d2, lq_new + i * M, bidx + i * M,
                          bidx_in ? bidx_in + i * M : NULL, NULL);
  }
  return bad ? ORA_E_NUMERIC : ORA_OK;
}
