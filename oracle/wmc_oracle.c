/*
 * wmc_oracle.c -- plain, slow, sequential CPU oracle for the signed-particle
 * Wigner Monte Carlo hot path (Sellier, Leygonie, Marceau Caron, "Combining
 * neural networks and signed particles to simulate quantum systems more
 * efficiently, Part II", arXiv:1806.00082).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant generator with the CUDA path.
 *
 * Everything is FP64 unless the method fixes another precision:
 *   - Wigner kernel: the discrete finite-window sum of Eq. (wigner-1d-discrete),
 *     summed over m = -h..h in ascending order, h = floor(L_C / (2 dx)).
 *   - gamma(x) = sum over M of V_W^+(x; M) (Eq. momentum_integral), and the
 *     CDF used to draw p' with probability V_W^+ / gamma (postulate, Sec. 2.1),
 *     both as exact sums of V_W^+ quantised to 62-bit fixed point relative to
 *     the row maximum (see wmco_cdf_row).
 *   - Particles follow the postulate of Sec. 2.1 (free drift, pair creation
 *     with probability gamma dt, children at p +- p') and rules 1 and 2
 *     (density from signed counts; annihilation of opposite signs in the same
 *     phase-space cell).
 *
 * Readings taken where the paper is silent (all listed in the design notes):
 *   cell i has centre (i + 1/2) dx; Delta k = pi / L_C, so the sine argument
 *   2 m dx j dp / hbar equals 2 pi (m j mod Q) / Q with Q = L_C / dx; V outside
 *   the domain is 0 (bc 0) or the edge value (bc 1); the momentum grid is
 *   M in [-n_M/2, n_M/2); children outside it are dropped (or wrapped); drift
 *   is f' = fl32(f + D[M]) on the within-cell offset f in [0, 1), with
 *   D[M] = fl32(M * hbar pi dt / (m Q dx^2)); after annihilation survivors are
 *   re-emitted row-major over (cell, M) with a fresh uniform offset; random
 *   numbers are Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) with key
 *   (seed_lo, seed_hi): particle id draws its offset from word id mod 4 of
 *   counter (id / 4, step, REPOS, sim), its pair-creation uniform u1 from word
 *   id mod 4 of (id / 4, step, GEN, sim) as a 32-bit fraction, and, only when
 *   a pair is created, p' from u53 of words 0, 1 of (id, step, PICK, sim).
 *
 * Build: gcc -O2 -ffp-contract=off -shared -fPIC (no FMA contraction, so the
 * FP32 drift is one rounded addition).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define WMCO_HBAR_EVS 6.582119569e-16 /* hbar [eV s] (CODATA 2018) */
#define WMCO_HBAR_JS 1.054571817e-34  /* hbar [J s]  (CODATA 2018) */
#define WMCO_PI 3.14159265358979323846

#define WMCO_PURPOSE_GEN 1u
#define WMCO_PURPOSE_REPOS 2u
#define WMCO_PURPOSE_PICK 3u

typedef struct {
  double dx_m;
  double mass_kg;
  double dt_s;
  uint64_t seed;
  int32_t n_x;
  int32_t Q;
  int32_t n_M;
  int32_t bc_potential;
  int32_t child_wrap;
  uint32_t sim;
} wmco_params;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, from its definition in Salmon et al., SC'11 (Sec. 3 and    */
/* Table 2): ten rounds of two 32x32->64 multiplications with the constants  */
/* 0xD2511F53 and 0xCD9E8D57, a word permutation, and a Weyl key schedule    */
/* with increments 0x9E3779B9 and 0xBB67AE85.                                */
/* ------------------------------------------------------------------------ */
void wmco_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform double in [0,1) from two words: 27 high bits of a, 26 of b. */
double wmco_u53(uint32_t a, uint32_t b) {
  return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6)) * (1.0 / 9007199254740992.0);
}

/* Uniform float in [0,1) on the 2^-24 grid from one word. */
float wmco_u24(uint32_t a) { return (float)(a >> 8) * (1.0f / 16777216.0f); }

/* Uniform double in [0,1) on the 2^-32 grid from one word. */
double wmco_u32(uint32_t a) { return (double)a * (1.0 / 4294967296.0); }

static void draw(const wmco_params* p, uint32_t c0, uint32_t step, uint32_t purpose, uint32_t out[4]) {
  uint32_t ctr[4] = {c0, step, purpose, p->sim};
  uint32_t key[2] = {(uint32_t)(p->seed & 0xffffffffu), (uint32_t)(p->seed >> 32)};
  wmco_philox4x32_10(ctr, key, out);
}

/* ------------------------------------------------------------------------ */
/* Wigner kernel, Eq. (wigner-1d-discrete)                                   */
/* ------------------------------------------------------------------------ */

/* sin(2 pi t / Q) for an integer t, by exact integer symmetry reduction so
 * that libm only ever sees an angle in [0, pi/4]. */
double wmco_sine(int32_t Q, int64_t t) {
  const int64_t h = Q / 2;
  int64_t r = t % Q;
  if (r < 0) r += Q;
  double sign = 1.0;
  if (r >= h) { r -= h; sign = -1.0; }          /* sin(x + pi) = -sin x   */
  if (2 * r > h) r = h - r;                      /* sin(pi - x) = sin x    */
  double v;
  if (4 * r > h)                                 /* sin x = cos(pi/2 - x)  */
    v = cos(WMCO_PI * (double)(h - 2 * r) / (double)(2 * h));
  else
    v = sin(WMCO_PI * (double)r / (double)h);
  return sign * v;
}

static double pot(const wmco_params* p, const double* V, int64_t l) {
  if (l >= 0 && l < p->n_x) return V[l];
  if (p->bc_potential == 0) return 0.0;
  return l < 0 ? V[0] : V[p->n_x - 1];
}

/* V_W(i; M) = -(dx / (hbar L_C)) sum_{m=-h}^{h} sin(2 m dx M dp / hbar) [V(i+m) - V(i-m)]
 *          = -(1 / (hbar Q))    sum_{m=-h}^{h} sin(2 pi m M / Q)   [V(i+m) - V(i-m)],
 * V in eV, result in 1/s.  One value. */
double wmco_kernel_value(const wmco_params* p, const double* V, int32_t i, int32_t M) {
  const int32_t h = p->Q / 2;
  double acc = 0.0;
  for (int32_t m = -h; m <= h; ++m) {
    double dV = pot(p, V, (int64_t)i + m) - pot(p, V, (int64_t)i - m);
    acc += wmco_sine(p->Q, (int64_t)m * (int64_t)M) * dV;
  }
  return -acc / (WMCO_HBAR_EVS * (double)p->Q);
}

/* Rows of the kernel over the momentum grid: out[r][k] = V_W(rows[r]; k - n_M/2).
 * The same sum as wmco_kernel_value, term by term and in the same order; the
 * Q sine values sin(2 pi t / Q) and the 2h + 1 differences of a row are
 * computed once and looked up, so every term is the identical FP64 product
 * and the result is bit-for-bit that of wmco_kernel_value. */
void wmco_kernel_rows(const wmco_params* p, const double* V, int32_t n_rows, const int32_t* rows,
                      double* out) {
  const int32_t Q = p->Q, h = Q / 2;
  double* S = (double*)malloc(sizeof(double) * (size_t)Q);
  double* dV = (double*)malloc(sizeof(double) * (size_t)(2 * h + 1));
  for (int32_t t = 0; t < Q; ++t) S[t] = wmco_sine(Q, t);
  for (int32_t r = 0; r < n_rows; ++r) {
    const int32_t i = rows[r];
    for (int32_t m = -h; m <= h; ++m) dV[m + h] = pot(p, V, (int64_t)i + m) - pot(p, V, (int64_t)i - m);
    for (int32_t k = 0; k < p->n_M; ++k) {
      const int64_t M = k - p->n_M / 2;
      const int64_t step = ((M % Q) + Q) % Q;          /* (m + 1) M - m M, reduced mod Q */
      int64_t t = (((int64_t)(-h) * M) % Q + Q) % Q;   /* (m M) mod Q at m = -h */
      double acc = 0.0;
      for (int32_t m = -h; m <= h; ++m) {
        acc += S[t] * dV[m + h];
        t += step;
        if (t >= Q) t -= Q;
      }
      out[(int64_t)r * p->n_M + k] = -acc / (WMCO_HBAR_EVS * (double)Q);
    }
  }
  free(S);
  free(dV);
}

/* Eq. (wigner-1d-discrete) by a sliding window instead of a sum per cell:
 * with E_M(l) = exp(i 2 pi l M / Q) the window sum is
 *   W_M(i) = sum_{l=i-h}^{i+h} V(l) E_M(l),   V_W(i; M) = -(2 / (hbar Q)) Im[ E_M(-i) W_M(i) ]
 * (the unfolded sum of the N = 1 network, sum_l V(l) sin((l - i) 2 pi M / Q)),
 * and W_M(i + 1) = W_M(i) + V(i + h + 1) E_M(i + h + 1) - V(i - h) E_M(i - h), so a
 * column costs O(n_x) instead of O(n_x h).  FP64 throughout, exact integer
 * phases (l M mod Q); V outside the domain follows bc_potential.  All cells:
 * out[i][k] = V_W(i; k - n_M/2), i = 0 .. n_x - 1.  An independent
 * arrangement of the same sum, to cross-check wmco_kernel_rows. */
void wmco_kernel_all_dft(const wmco_params* p, const double* V, double* out) {
  const int32_t Q = p->Q, h = Q / 2;
  const int64_t nx = p->n_x;
  double* C = (double*)malloc(sizeof(double) * (size_t)Q);
  double* S = (double*)malloc(sizeof(double) * (size_t)Q);
  /* sin(2 pi t / Q), and cos(2 pi t / Q) = sin(2 pi (4t + Q) / (4Q)) */
  for (int32_t t = 0; t < Q; ++t) {
    S[t] = wmco_sine(Q, t);
    C[t] = wmco_sine(4 * Q, 4 * (int64_t)t + Q);
  }
  for (int32_t k = 0; k < p->n_M; ++k) {
    const int64_t M = k - p->n_M / 2;
    const int64_t Mq = ((M % Q) + Q) % Q;
    double wr = 0.0, wi = 0.0;                   /* W_M(0) */
    for (int64_t l = -h; l <= h; ++l) {
      const int64_t t = ((l * Mq) % Q + Q) % Q;
      const double v = pot(p, V, l);
      wr += v * C[t];
      wi += v * S[t];
    }
    for (int64_t i = 0; i < nx; ++i) {
      const int64_t ti = ((i * Mq) % Q + Q) % Q;  /* E_M(-i) = C[ti] - i S[ti] */
      out[i * p->n_M + k] = -(2.0 / (WMCO_HBAR_EVS * (double)Q)) * (C[ti] * wi - S[ti] * wr);
      const int64_t la = i + h + 1, lb = i - h;
      const int64_t ta = ((la * Mq) % Q + Q) % Q, tb = ((lb * Mq) % Q + Q) % Q;
      const double va = pot(p, V, la), vb = pot(p, V, lb);
      wr += va * C[ta] - vb * C[tb];
      wi += va * S[ta] - vb * S[tb];
    }
  }
  free(C);
  free(S);
}

/* The N = 2 network of Eq. (kernel_ML) with the barycentric weights of Sec. 2.3
 * (omega^V = (1, 1), omega^theta = (1/2, 1/2), W_l = w_l = -2 dx / (hbar L_C),
 * one cosine factor since N = 2^1): the terms V(l) sin(theta_l(i, j)) of the
 * N = 1 network are grouped by consecutive cells (2q, 2q + 1), V is replaced by
 * the pair's average and sin a + sin b = 2 sin((a + b)/2) cos((a - b)/2), so
 *   V_W2(i; M) = -(2 / (hbar Q)) cos(pi M / Q)
 *                sum_{q: i-h <= 2q, 2q+1 <= i+h} [V(2q) + V(2q+1)] sin(pi (4q + 1 - 2i) M / Q),
 * theta_l(i, j) = (l - i) 2 pi M / Q.  The pairs lie inside the window
 * [i - h, i + h]; the one cell of the window left out has a zero sine.
 * Sines of the period-2Q integer phases sin(2 pi t / (2Q)), t exact mod 2Q. */
void wmco_kernel_rows_n2(const wmco_params* p, const double* V, int32_t n_rows, const int32_t* rows,
                         double* out) {
  const int32_t Q = p->Q, h = Q / 2, Q2 = 2 * Q;
  double* S2 = (double*)malloc(sizeof(double) * (size_t)Q2);
  for (int32_t t = 0; t < Q2; ++t) S2[t] = wmco_sine(Q2, t);
  for (int32_t r = 0; r < n_rows; ++r) {
    const int64_t i = rows[r];
    /* first pair: the smallest even 2q >= i - h */
    int64_t q0 = i - h;
    if (q0 % 2 != 0) q0 += 1;            /* (works for negative q0 as well: |q0 % 2| = 1) */
    for (int32_t k = 0; k < p->n_M; ++k) {
      const int64_t M = k - p->n_M / 2;
      double acc = 0.0;
      for (int64_t l = q0; l + 1 <= i + h; l += 2) {
        int64_t t = ((2 * (l - i) + 1) * M) % Q2;
        if (t < 0) t += Q2;
        acc += (pot(p, V, l) + pot(p, V, l + 1)) * S2[t];
      }
      int64_t tc = (M + h) % Q2;          /* cos(pi M / Q) = sin(2 pi (M + Q/2) / (2Q)) */
      if (tc < 0) tc += Q2;
      out[(int64_t)r * p->n_M + k] = -(2.0 / (WMCO_HBAR_EVS * (double)Q)) * S2[tc] * acc;
    }
  }
  free(S2);
}

/* Smallest L with 2^L >= n. */
static int32_t ceil_log2(int32_t n) {
  int32_t L = 0;
  while ((1 << L) < n) ++L;
  return L;
}

/* gamma and the momentum CDF of one kernel row (Eq. momentum_integral and the
 * postulate's p' ~ V_W^+ / gamma).  The positive parts x_k = max(V_W[k], 0)
 * are quantised to integers relative to the row maximum,
 *   e = floor(log2(max_k x_k)),  s = 61 - ceil(log2(n_M)) - e,
 *   q_k = x_k 2^s rounded to the nearest integer (ties to even),
 * so that every q_k < 2^(62 - ceil(log2 n_M)) and their sum fits 62 bits; the
 * CDF is the exact running sum cdf[k] = sum_{k' <= k} q_k', the row total is
 * Qtot = cdf[n_M - 1], and gamma = fl64(Qtot 2^-s).  A row with no positive
 * entry has gamma = 0 and a zero CDF.  *scale receives s.  Returns gamma. */
double wmco_cdf_row(int32_t n_M, const double* vw, int64_t* cdf, int32_t* scale) {
  double xmax = 0.0;
  for (int32_t k = 0; k < n_M; ++k)
    if (vw[k] > xmax) xmax = vw[k];
  if (xmax == 0.0) {
    for (int32_t k = 0; k < n_M; ++k) cdf[k] = 0;
    if (scale) *scale = 0;
    return 0.0;
  }
  int fe;
  frexp(xmax, &fe);                 /* xmax = f 2^fe, f in [1/2, 1) */
  const int32_t e = fe - 1;
  const int32_t s = 61 - ceil_log2(n_M) - e;
  int64_t run = 0;
  for (int32_t k = 0; k < n_M; ++k) {
    const double x = vw[k] > 0.0 ? vw[k] : 0.0;
    run += (int64_t)rint(ldexp(x, s)); /* exact scaling, round half to even */
    cdf[k] = run;
  }
  if (scale) *scale = s;
  return ldexp((double)run, -s);
}

/* Index k of p' drawn from V_W^+ / gamma with the 53-bit uniform integer U2:
 * target = floor(U2 Qtot / 2^53) < Qtot, and k is the smallest index with
 * cdf[k] > target (it always exists). */
int32_t wmco_sample_row(int32_t n_M, const int64_t* cdf, uint64_t U2) {
  const unsigned __int128 prod = (unsigned __int128)U2 * (unsigned __int128)(uint64_t)cdf[n_M - 1];
  const int64_t target = (int64_t)(prod >> 53);
  for (int32_t k = 0; k < n_M; ++k)
    if (cdf[k] > target) return k;
  return -1;
}

/* The 53-bit integer behind wmco_u53(a, b). */
uint64_t wmco_u53_bits(uint32_t a, uint32_t b) { return ((uint64_t)(a >> 5) << 26) | (uint64_t)(b >> 6); }

/* Drift per step in cells, D[M] = fl32(M * hbar pi dt / (m Q dx^2)). */
void wmco_drift_table(const wmco_params* p, float* D) {
  double d1 = ((WMCO_HBAR_JS * WMCO_PI) * p->dt_s) / ((p->mass_kg * (double)p->Q) * (p->dx_m * p->dx_m));
  for (int32_t k = 0; k < p->n_M; ++k) D[k] = (float)((double)(k - p->n_M / 2) * d1);
}

/* ------------------------------------------------------------------------ */
/* Ensemble: rebuild (rule 2 survivors), step (postulate), density (rule 1) */
/* ------------------------------------------------------------------------ */

typedef struct {
  int64_t n;
  int32_t* cell;
  float* f;
  int16_t* M;
  int8_t* s;
} ensemble;

static void ens_free(ensemble* e) {
  free(e->cell); free(e->f); free(e->M); free(e->s);
  memset(e, 0, sizeof(*e));
}

/* Population of a signed histogram: sum of |n(i, M)|. */
int64_t wmco_population(const wmco_params* p, const int32_t* hist) {
  int64_t P = 0;
  for (int64_t q = 0; q < (int64_t)p->n_x * p->n_M; ++q) P += hist[q] < 0 ? -(int64_t)hist[q] : hist[q];
  return P;
}

/* Survivors of a net signed histogram, in row-major (cell, M) order, each
 * with a fresh offset f = u24(word id mod 4 of Philox(id / 4, step, REPOS, sim)),
 * where the particle's number id is id_base plus its place in this histogram
 * (id_base = 0 for a whole domain; a sub-domain of cells numbers its particles
 * after those of the cells before it).  Outputs are indexed by the place.
 * Returns the count written, or -1 if it exceeds capacity or the ids 2^32. */
static int64_t materialize_from(const wmco_params* p, const int32_t* hist, uint32_t step, int64_t capacity,
                                uint64_t id_base, int32_t* cell, float* f, int16_t* M, int8_t* s) {
  int64_t id = 0;
  for (int32_t i = 0; i < p->n_x; ++i) {
    for (int32_t k = 0; k < p->n_M; ++k) {
      int32_t n = hist[(int64_t)i * p->n_M + k];
      int32_t a = n < 0 ? -n : n;
      for (int32_t c = 0; c < a; ++c) {
        const uint64_t gid = id_base + (uint64_t)id;
        if (id >= capacity || gid >= ((uint64_t)1 << 32)) return -1;
        uint32_t w[4];
        draw(p, (uint32_t)(gid >> 2), step, WMCO_PURPOSE_REPOS, w);
        cell[id] = i;
        f[id] = wmco_u24(w[gid & 3]);
        M[id] = (int16_t)(k - p->n_M / 2);
        s[id] = (int8_t)(n > 0 ? 1 : -1);
        ++id;
      }
    }
  }
  return id;
}

int64_t wmco_materialize(const wmco_params* p, const int32_t* hist, uint32_t step, int64_t capacity,
                         int32_t* cell, float* f, int16_t* M, int8_t* s) {
  return materialize_from(p, hist, step, capacity, 0u, cell, f, M, s);
}

/* Rule 1: rho(i) = sum over M of the signed counts. */
void wmco_density(const wmco_params* p, const int32_t* hist, int64_t* rho) {
  for (int32_t i = 0; i < p->n_x; ++i) {
    int64_t a = 0;
    for (int32_t k = 0; k < p->n_M; ++k) a += hist[(int64_t)i * p->n_M + k];
    rho[i] = a;
  }
}

enum {
  ST_PAIRS = 0,          /* pairs created                                  */
  ST_ABSORBED = 1,       /* particles that left [0, n_x)                   */
  ST_ABSORBED_SIGNED = 2,/* sum of their signs                             */
  ST_DROPPED = 3,        /* children outside the momentum grid             */
  ST_DROPPED_SIGNED = 4, /* sum of their signs                             */
  ST_RATE = 5,           /* evaluated cells with gamma dt >= 1             */
  ST_POP = 6,            /* population after the last step                 */
  ST_NET = 7,            /* net sign after the last step                   */
  ST_PARTICLE_STEPS = 8, /* sum over steps of the population at step start */
  ST_ERR = 9,            /* 0 ok; 1 capacity; 2 drift of a cell or more    */
  ST_N = 10
};

/* Run n_steps steps t = t_first, ..., t_first + n_steps - 1 on the net
 * histogram hist (the state after the rebuild of step t_first - 1), writing
 * the net histogram after the last step into hist_out.
 *
 * table: NULL to evaluate Eq. (wigner-1d-discrete) in FP64 on the occupied
 * cells each step, or a full FP32 table [n_x][n_M] of V_W used instead (so
 * that two implementations can be fed the same kernel values).
 * V: potential [n_x] in eV (ignored if table is given).
 * stats: int64[ST_N], accumulated. Returns 0 or an ST_ERR code. */
static int32_t simulate_from(const wmco_params* p, const double* V, const float* table, const int32_t* hist,
                             uint32_t t_first, int32_t n_steps, uint64_t id_base, int32_t* hist_out,
                             int64_t* stats);

int32_t wmco_simulate(const wmco_params* p, const double* V, const float* table, const int32_t* hist,
                      uint32_t t_first, int32_t n_steps, int32_t* hist_out, int64_t* stats) {
  return simulate_from(p, V, table, hist, t_first, n_steps, 0u, hist_out, stats);
}

/* One step of a sub-domain of cells (its particles only in hist; every other
 * row zero), its particles numbered from id_base: the particles of the cells
 * before it in a domain decomposition come first.  Particles that drift out of
 * the sub-domain land in the neighbouring rows of hist_out (to be passed to
 * the rank that owns them); only leaving [0, n_x) absorbs. */
int32_t wmco_simulate_subdomain(const wmco_params* p, const double* V, const float* table, const int32_t* hist,
                                uint32_t t, uint64_t id_base, int32_t* hist_out, int64_t* stats) {
  return simulate_from(p, V, table, hist, t, 1, id_base, hist_out, stats);
}

static int32_t simulate_from(const wmco_params* p, const double* V, const float* table, const int32_t* hist,
                             uint32_t t_first, int32_t n_steps, uint64_t id_base, int32_t* hist_out,
                             int64_t* stats) {
  const int64_t nx = p->n_x, nM = p->n_M, G = nx * nM;
  float* D = (float*)malloc(sizeof(float) * nM);
  wmco_drift_table(p, D);
  for (int64_t k = 0; k < nM; ++k)
    if (!(fabsf(D[k]) < 1.0f)) { free(D); stats[ST_ERR] = 2; return 2; }

  int32_t* cur = (int32_t*)malloc(sizeof(int32_t) * G);
  int64_t* acc = (int64_t*)malloc(sizeof(int64_t) * G);
  memcpy(cur, hist, sizeof(int32_t) * G);
  double* vw = (double*)malloc(sizeof(double) * G);   /* rows computed on demand */
  int64_t* cdf = (int64_t*)malloc(sizeof(int64_t) * G);
  double* gam = (double*)malloc(sizeof(double) * nx);
  char* have = (char*)malloc(nx);
  int32_t err = 0;

  for (int32_t st = 0; st < n_steps && !err; ++st) {
    const uint32_t t = t_first + (uint32_t)st;
    /* survivors of the previous step, re-emitted at step t - 1 */
    int64_t P = wmco_population(p, cur);
    ensemble e = {0};
    e.cell = (int32_t*)malloc(sizeof(int32_t) * (P ? P : 1));
    e.f = (float*)malloc(sizeof(float) * (P ? P : 1));
    e.M = (int16_t*)malloc(sizeof(int16_t) * (P ? P : 1));
    e.s = (int8_t*)malloc(P ? P : 1);
    e.n = materialize_from(p, cur, t - 1u, P, id_base, e.cell, e.f, e.M, e.s);
    if (e.n < 0) { err = 1; ens_free(&e); break; }
    stats[ST_PARTICLE_STEPS] += e.n;

    memset(acc, 0, sizeof(int64_t) * G);
    memset(have, 0, nx);
    for (int64_t id = 0; id < e.n; ++id) {
      const int32_t k = e.M[id] + p->n_M / 2;
      const int32_t sgn = e.s[id];
      /* free drift of the within-cell offset (one FP32 rounding) */
      float fn = e.f[id] + D[k];
      int32_t c = e.cell[id] + (fn >= 1.0f ? 1 : (fn < 0.0f ? -1 : 0));
      if (c < 0 || c >= p->n_x) {
        stats[ST_ABSORBED] += 1;
        stats[ST_ABSORBED_SIGNED] += sgn;
        continue;
      }
      /* kernel on an occupied cell, evaluated when first needed this step */
      double* row = vw + (int64_t)c * nM;
      int64_t* crow = cdf + (int64_t)c * nM;
      if (!have[c]) {
        if (table) {
          for (int64_t q = 0; q < nM; ++q) row[q] = (double)table[(int64_t)c * nM + q];
        } else {
          wmco_kernel_rows(p, V, 1, &c, row);
        }
        gam[c] = wmco_cdf_row(p->n_M, row, crow, NULL);
        if (gam[c] * p->dt_s >= 1.0) stats[ST_RATE] += 1;
        have[c] = 1;
      }
      /* pair creation with probability gamma dt */
      uint32_t w[4];
      const uint64_t gid = id_base + (uint64_t)id;
      draw(p, (uint32_t)(gid >> 2), t, WMCO_PURPOSE_GEN, w);
      double u1 = wmco_u32(w[gid & 3]);
      if (u1 < gam[c] * p->dt_s) {
        draw(p, (uint32_t)gid, t, WMCO_PURPOSE_PICK, w);
        int32_t kp = wmco_sample_row(p->n_M, crow, wmco_u53_bits(w[0], w[1]));
        int32_t Mp = kp - p->n_M / 2;
        int32_t Mc[2] = {e.M[id] + Mp, e.M[id] - Mp};
        int32_t sc[2] = {sgn, -sgn};
        stats[ST_PAIRS] += 1;
        for (int q = 0; q < 2; ++q) {
          int32_t kc = Mc[q] + p->n_M / 2;
          if (kc < 0 || kc >= p->n_M) {
            if (!p->child_wrap) {
              stats[ST_DROPPED] += 1;
              stats[ST_DROPPED_SIGNED] += sc[q];
              continue;
            }
            kc = ((kc % p->n_M) + p->n_M) % p->n_M;
          }
          acc[(int64_t)c * nM + kc] += sc[q];
        }
      }
      /* the parent keeps its momentum */
      acc[(int64_t)c * nM + k] += sgn;
    }
    ens_free(&e);
    /* rule 2: opposite signs in one (cell, M) cancel; the net count survives */
    for (int64_t q = 0; q < G; ++q) {
      if (acc[q] > INT32_MAX || acc[q] < -INT32_MAX) { err = 1; break; }
      cur[q] = (int32_t)acc[q];
    }
  }
  if (!err) {
    memcpy(hist_out, cur, sizeof(int32_t) * G);
    int64_t pop = 0, net = 0;
    for (int64_t q = 0; q < G; ++q) { pop += cur[q] < 0 ? -(int64_t)cur[q] : cur[q]; net += cur[q]; }
    stats[ST_POP] = pop;
    stats[ST_NET] = net;
  }
  stats[ST_ERR] = err;
  free(D); free(cur); free(acc); free(vw); free(cdf); free(gam); free(have);
  return err;
}
