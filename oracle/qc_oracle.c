/*
 * CPU oracle for the full state-vector simulation defined in QCLAB
 * (Keip, Camps, Van Beeumen, "QCLAB: A Matlab Toolbox for Quantum Computing",
 * arXiv:2503.03016, 2025).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares no source, header,
 * table or helper with the CUDA path, and the CUDA path never calls it.
 *
 * Everything is plain complex128 (interleaved re, im doubles), one gate per pass,
 * written straight from the definitions:
 *
 *  - Sec. 3.2: a gate U' on some qubits acts on the register as I_l (x) U' (x) I_r.
 *    With qubit 0 the most significant index bit (Sec. 5.1: kron(v, bell) puts v on
 *    q0), qubit q is bit n-1-q of the amplitude index.  Applying I_l (x) U' (x) I_r
 *    without forming the matrix means: for every index with the gate's bits clear,
 *    gather the 2^k amplitudes that differ only in those bits and multiply them by U'.
 *  - Sec. 3.3: P(|0>) = sum of |psi_i|^2 over indices whose measured bit is 0; the
 *    collapsed state keeps that half and divides it by sqrt(P).
 *
 * Compiled with -ffp-contract=off so that no multiply-add is fused behind the
 * reader's back; |a|^2 = re*re + im*im is then two rounded products and one
 * rounded sum, as the sampling convention requires.
 *
 * Parity pins for every function live in tests/test_oracle_pins.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define RE(p, i) ((p)[2 * (i)])
#define IM(p, i) ((p)[2 * (i) + 1])

/* c = a * b for complex numbers given as (re, im) */
static inline void cmul(double ar, double ai, double br, double bi, double* cr, double* ci) {
  *cr = ar * br - ai * bi;
  *ci = ar * bi + ai * br;
}

static inline uint64_t qbit(int n, int q) { return (uint64_t)1 << (n - 1 - q); }

/* Dense single-qubit gate.  U is row-major 2x2, (re, im) pairs. */
void orc_apply_1q(double* psi, int n, int q, const double* U) {
  const int64_t N = (int64_t)1 << n;
  const uint64_t m = qbit(n, q);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < N; ++i) {
    if ((uint64_t)i & m) continue;
    const int64_t j = (int64_t)((uint64_t)i | m);
    double a0r = RE(psi, i), a0i = IM(psi, i), a1r = RE(psi, j), a1i = IM(psi, j);
    double t0r, t0i, t1r, t1i;
    cmul(U[0], U[1], a0r, a0i, &t0r, &t0i);
    cmul(U[2], U[3], a1r, a1i, &t1r, &t1i);
    double o0r = t0r + t1r, o0i = t0i + t1i;
    cmul(U[4], U[5], a0r, a0i, &t0r, &t0i);
    cmul(U[6], U[7], a1r, a1i, &t1r, &t1i);
    RE(psi, i) = o0r;
    IM(psi, i) = o0i;
    RE(psi, j) = t0r + t1r;
    IM(psi, j) = t0i + t1i;
  }
}

/*
 * Dense gate on k distinct qubits (any order, any positions).  U is row-major
 * 2^k x 2^k; its row/column index r has qubits[0] as the most significant bit,
 * i.e. U acts on the kron-ordered factor qubits[0] (x) qubits[1] (x) ... .
 */
void orc_apply_kq(double* psi, int n, const int* qubits, int k, const double* U) {
  const int64_t N = (int64_t)1 << n;
  const int64_t D = (int64_t)1 << k;
  uint64_t all = 0;
  for (int j = 0; j < k; ++j) all |= qbit(n, qubits[j]);
#pragma omp parallel
  {
    int64_t* idx = (int64_t*)malloc(sizeof(int64_t) * D);
    double* v = (double*)malloc(sizeof(double) * 2 * D);
#pragma omp for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
      if ((uint64_t)i & all) continue;
      for (int64_t r = 0; r < D; ++r) {
        uint64_t x = (uint64_t)i;
        for (int j = 0; j < k; ++j)
          if ((r >> (k - 1 - j)) & 1) x |= qbit(n, qubits[j]);
        idx[r] = (int64_t)x;
        v[2 * r] = RE(psi, x);
        v[2 * r + 1] = IM(psi, x);
      }
      for (int64_t r = 0; r < D; ++r) {
        double sr = 0.0, si = 0.0;
        for (int64_t c = 0; c < D; ++c) {
          double tr, ti;
          cmul(U[2 * (r * D + c)], U[2 * (r * D + c) + 1], v[2 * c], v[2 * c + 1], &tr, &ti);
          sr += tr;
          si += ti;
        }
        RE(psi, idx[r]) = sr;
        IM(psi, idx[r]) = si;
      }
    }
    free(idx);
    free(v);
  }
}

/* Dense two-qubit gate; row index = 2*b_qa + b_qb (qa is the first kron factor). */
void orc_apply_2q(double* psi, int n, int qa, int qb, const double* U) {
  int qs[2] = {qa, qb};
  orc_apply_kq(psi, n, qs, 2, U);
}

/*
 * Single-qubit U on `target`, applied only on indices whose control bits equal the
 * requested states (states[j] in {0,1}; state 0 is the open control drawn in the
 * error-correction example of Sec. 5.4).
 */
void orc_apply_ctrl(double* psi, int n, const int* ctrls, const int* states, int nctrl, int target,
                    const double* U) {
  const int64_t N = (int64_t)1 << n;
  const uint64_t m = qbit(n, target);
  uint64_t cmask = 0, cval = 0;
  for (int j = 0; j < nctrl; ++j) {
    cmask |= qbit(n, ctrls[j]);
    if (states[j]) cval |= qbit(n, ctrls[j]);
  }
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < N; ++i) {
    if ((uint64_t)i & m) continue;
    if (((uint64_t)i & cmask) != cval) continue;
    const int64_t j = (int64_t)((uint64_t)i | m);
    double a0r = RE(psi, i), a0i = IM(psi, i), a1r = RE(psi, j), a1i = IM(psi, j);
    double t0r, t0i, t1r, t1i;
    cmul(U[0], U[1], a0r, a0i, &t0r, &t0i);
    cmul(U[2], U[3], a1r, a1i, &t1r, &t1i);
    double o0r = t0r + t1r, o0i = t0i + t1i;
    cmul(U[4], U[5], a0r, a0i, &t0r, &t0i);
    cmul(U[6], U[7], a1r, a1i, &t1r, &t1i);
    RE(psi, i) = o0r;
    IM(psi, i) = o0i;
    RE(psi, j) = t0r + t1r;
    IM(psi, j) = t0i + t1i;
  }
}

/* p_i = re*re + im*im (two rounded products, one rounded sum). */
void orc_probs(const double* psi, int n, double* p) {
  const int64_t N = (int64_t)1 << n;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < N; ++i) {
    double a = RE(psi, i) * RE(psi, i);
    double b = IM(psi, i) * IM(psi, i);
    p[i] = a + b;
  }
}

/* Sec. 3.3: P(outcome) = sum over indices whose bit for qubit q equals outcome. */
double orc_outcome_prob(const double* psi, int n, int q, int outcome) {
  const int64_t N = (int64_t)1 << n;
  const uint64_t m = qbit(n, q);
  double s = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : s)
  for (int64_t i = 0; i < N; ++i) {
    int b = ((uint64_t)i & m) ? 1 : 0;
    if (b != outcome) continue;
    double a = RE(psi, i) * RE(psi, i);
    double c = IM(psi, i) * IM(psi, i);
    s += a + c;
  }
  return s;
}

/* Sec. 3.3: keep the `outcome` half, zero the other, divide by sqrt(P). */
void orc_collapse(double* psi, int n, int q, int outcome, double P) {
  const int64_t N = (int64_t)1 << n;
  const uint64_t m = qbit(n, q);
  const double s = sqrt(P);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < N; ++i) {
    int b = ((uint64_t)i & m) ? 1 : 0;
    if (b != outcome) {
      RE(psi, i) = 0.0;
      IM(psi, i) = 0.0;
    } else {
      RE(psi, i) = RE(psi, i) / s;
      IM(psi, i) = IM(psi, i) / s;
    }
  }
}

/*
 * Cumulative distribution cdf_k = sum_{i<=k} p_i, accumulated sequentially in
 * double-double (TwoSum of Knuth, TAOCP vol. 2; Fast2Sum of Dekker 1971) and rounded
 * once per entry, so that cdf_k is the FP64 number nearest to the exact prefix sum.
 */
void orc_cdf(const double* p, int64_t N, double* cdf) {
  double hi = 0.0, lo = 0.0;
  for (int64_t i = 0; i < N; ++i) {
    /* (s, e) = TwoSum(hi, p_i) */
    double s = hi + p[i];
    double bb = s - hi;
    double e = (hi - (s - bb)) + (p[i] - bb);
    e += lo;
    /* (hi, lo) = Fast2Sum(s, e) */
    hi = s + e;
    lo = e - (hi - s);
    cdf[i] = hi;
  }
}

/* outcome(u) = min{k : u*T < cdf_k}, T = cdf_{N-1}; found by bisection. */
void orc_sample(const double* cdf, int64_t N, const double* u, int64_t shots, uint64_t* out) {
  const double T = cdf[N - 1];
#pragma omp parallel for schedule(static)
  for (int64_t s = 0; s < shots; ++s) {
    const double t = u[s] * T;
    int64_t lo = 0, hi = N - 1; /* answer in [lo, hi]; cdf[N-1] = T > t for u < 1 */
    while (lo < hi) {
      int64_t mid = lo + (hi - lo) / 2;
      if (t < cdf[mid])
        hi = mid;
      else
        lo = mid + 1;
    }
    out[s] = (uint64_t)lo;
  }
}

/* <a|b> = sum_i conj(a_i) b_i */
void orc_inner(const double* a, const double* b, int64_t N, double* out) {
  double sr = 0.0, si = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : sr, si)
  for (int64_t i = 0; i < N; ++i) {
    double tr, ti;
    cmul(RE(a, i), -IM(a, i), RE(b, i), IM(b, i), &tr, &ti);
    sr += tr;
    si += ti;
  }
  out[0] = sr;
  out[1] = si;
}

/*
 * <psi| P |psi> for a Pauli term given by index-bit masks (x, z): P acts on the
 * qubit of index bit b as X if only x has bit b, Z if only z has it, Y if both, so
 * P = i^{|x & z|} X^x Z^z (Y = iXZ) and P|j> = i^{|x & z|} (-1)^{|j & z|} |j ^ x>.
 * Hence <psi|P|psi> = i^{|x & z|} sum_j conj(psi_{j^x}) (-1)^{|j & z|} psi_j, written
 * out term by term (Sec. 5.2 estimates a density matrix from such expectations).
 * out = (re, im); the imaginary part is zero up to rounding for a Hermitian P.
 */
void orc_expect_masks(const double* psi, int n, uint64_t x, uint64_t z, double* out) {
  const int64_t N = (int64_t)1 << n;
  double sr = 0.0, si = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : sr, si)
  for (int64_t j = 0; j < N; ++j) {
    const int64_t k = (int64_t)((uint64_t)j ^ x);
    const double sgn = (__builtin_popcountll((uint64_t)j & z) & 1) ? -1.0 : 1.0;
    double tr, ti;
    cmul(RE(psi, k), -IM(psi, k), RE(psi, j), IM(psi, j), &tr, &ti);
    sr += sgn * tr;
    si += sgn * ti;
  }
  /* multiply by i^{|x & z|} */
  const int ny = __builtin_popcountll(x & z) & 3;
  double r = sr, i = si;
  for (int t = 0; t < ny; ++t) {
    const double nr = -i;
    i = r;
    r = nr;
  }
  out[0] = r;
  out[1] = i;
}

/* ---------------------------------------------------------------------------
 * Seeded start states regenerated from the amplitude index (so that 2^32-amplitude
 * states need no host copy).  SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) used as a
 * counter-based stream: output c = mix(seed + (c+1)*gamma).  Amplitude j takes
 * u1 = U(2j), u2 = U(2j+1) and the Box-Muller transform.
 * ------------------------------------------------------------------------- */
static inline uint64_t sm64(uint64_t seed, uint64_t c) {
  uint64_t z = seed + (c + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
static inline double sm_uniform(uint64_t seed, uint64_t c) {
  return (double)(sm64(seed, c) >> 11) * 0x1.0p-53;
}
static inline void gauss_amp(uint64_t seed, uint64_t j, double* re, double* im) {
  double u1 = sm_uniform(seed, 2 * j), u2 = sm_uniform(seed, 2 * j + 1);
  double r = sqrt(-2.0 * log1p(-u1));
  double t = 2.0 * M_PI * u2;
  *re = r * cos(t);
  *im = r * sin(t);
}

void orc_gaussian_amplitudes(uint64_t seed, int64_t start, int64_t count, double* out) {
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < count; ++j) gauss_amp(seed, (uint64_t)(start + j), &out[2 * j], &out[2 * j + 1]);
}

/* sum_j |x_j|^2 of the unnormalised Gaussian state */
double orc_gaussian_norm2(uint64_t seed, int n) {
  const int64_t N = (int64_t)1 << n;
  double s = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : s)
  for (int64_t j = 0; j < N; ++j) {
    double re, im;
    gauss_amp(seed, (uint64_t)j, &re, &im);
    double a = re * re;
    double b = im * im;
    s += a + b;
  }
  return s;
}

/*
 * Discrete Fourier transform of the normalised Gaussian state at chosen output
 * indices: y_k = N^{-1/2} sum_j x_j exp(+2 pi i j k / N), x_j = g_j / sqrt(norm2).
 * The phase uses the exact integer (j*k mod N), so each term is exp(2 pi i r / N)
 * with r < N.  If round_c64 is set, x_j is rounded to single precision first
 * (the complex64 start state).  This is the closed form the quantum Fourier
 * transform circuit must reproduce (qubit 0 = most significant bit).
 */
void orc_dft_gaussian(uint64_t seed, int n, double norm2, int round_c64, const uint64_t* ks, int nk,
                      double* out) {
  const int64_t N = (int64_t)1 << n;
  const uint64_t mask = (uint64_t)N - 1;
  const double inv = 1.0 / sqrt(norm2);
  for (int t = 0; t < 2 * nk; ++t) out[t] = 0.0;
  /* one pass over j (each amplitude generated once); per-thread partial sums over a
   * contiguous range of j, added in thread order at the end */
#pragma omp parallel
  {
    double* acc = (double*)calloc((size_t)(2 * nk), sizeof(double));
#pragma omp for schedule(static)
    for (int64_t j = 0; j < N; ++j) {
      double re, im;
      gauss_amp(seed, (uint64_t)j, &re, &im);
      re = re * inv;
      im = im * inv;
      if (round_c64) {
        re = (double)(float)re;
        im = (double)(float)im;
      }
      for (int t = 0; t < nk; ++t) {
        uint64_t r = ((uint64_t)j * ks[t]) & mask;
        double ang = 2.0 * M_PI * ((double)r / (double)N);
        double tr, ti;
        cmul(re, im, cos(ang), sin(ang), &tr, &ti);
        acc[2 * t] += tr;
        acc[2 * t + 1] += ti;
      }
    }
#pragma omp for ordered schedule(static, 1)
    for (int th = 0; th < omp_get_num_threads(); ++th) {
#pragma omp ordered
      for (int t = 0; t < 2 * nk; ++t) out[t] += acc[t];
    }
    free(acc);
  }
  const double sc = 1.0 / sqrt((double)N);
  for (int t = 0; t < 2 * nk; ++t) out[t] *= sc;
}

/* thread count of the parallel loops (timing of the CPU baseline; results do not
 * depend on it except for the summation order of reductions) */
void orc_set_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
#else
  (void)t;
#endif
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
