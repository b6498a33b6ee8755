/*
 * FP64 CPU oracle of OCD soft-output detection in plain C, one subcarrier per
 * OpenMP iteration.
 *
 * TEST INFRASTRUCTURE ONLY.  It restates the same steps as the NumPy oracle
 * (oracle/ocd.py) as scalar loops, so that the CPU baseline can use every
 * host core; the test-suite checks the two against each other.  It shares no
 * code with the CUDA library and the library never calls it.
 *
 * Wu, Dick, Cavallaro, Studer, "High-Throughput Data Detection for Massive
 * MU-MIMO-OFDM using Coordinate Descent" (arXiv 1611.08779):
 *   - Algorithm 1: preprocessing (||h_u||^2, d_u^-1 = (||h_u||^2 + alpha)^-1,
 *     p_u = d_u^-1 ||h_u||^2), then K round-robin sweeps over the users with
 *     the residual r = y - H z kept up to date (Eq. 15);
 *   - Eq. 14 and the QAM / BPSK cases after it: projection onto the box;
 *   - Eq. 9 with the approximation of Section III-C: max-log LLRs with
 *     mu~ = p_u and rho~ = ||h_u||^2 Es / N0, minima over the whole alphabet.
 * The readings (general Es, BOX-mode rho~, Gray labelling, the LLR sign, a
 * zero column) are the NumPy oracle's.
 *
 * Layouts, interleaved (re, im) doubles, row-major:
 *   H [Nsc][B][U], Y [Nsc][T][B], z [Nsc][T][U], llr [Nsc][T][U][Q] (doubles).
 * Compiled with -ffp-contract=off so that no multiply-add is fused and the
 * result does not depend on the host's instruction set.
 */
#include <math.h>
#include <stddef.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAX_B 512
#define ORC_MAX_U 32
#define ORC_MAX_POINTS 256
#define ORC_MAX_Q 8

/* Gray word of level index i (binary-reflected). */
static int gray(int i) { return i ^ (i >> 1); }

/*
 * Unit-energy alphabet and its labels (Section II-A): level index i of
 * M = sqrt(|O|) has amplitude (2i - (M-1)) / sigma, sigma^2 = 2 (M^2 - 1) / 3;
 * the first Q/2 label bits (MSB first) are the Gray word of the in-phase
 * level, the next Q/2 that of the quadrature level.  BPSK: {-1, +1} with
 * labels 0, 1.  Returns the number of points, or 0 for an unknown order.
 */
static int alphabet(int order, double* re, double* im, unsigned char lab[][ORC_MAX_Q], int* Q) {
  if (order == 2) {
    re[0] = -1.0; im[0] = 0.0; lab[0][0] = 0;
    re[1] = 1.0; im[1] = 0.0; lab[1][0] = 1;
    *Q = 1;
    return 2;
  }
  int q;
  switch (order) {
    case 4: q = 2; break;
    case 16: q = 4; break;
    case 64: q = 6; break;
    case 256: q = 8; break;
    default: return 0;
  }
  const int half = q / 2;
  const int M = 1 << half;
  const double sigma = sqrt(2.0 * (double)(M * M - 1) / 3.0);
  int n = 0;
  for (int ii = 0; ii < M; ++ii)
    for (int iq = 0; iq < M; ++iq) {
      re[n] = (double)(2 * ii - (M - 1)) / sigma;
      im[n] = (double)(2 * iq - (M - 1)) / sigma;
      const int word = (gray(ii) << half) | gray(iq);
      for (int b = 0; b < q; ++b) lab[n][b] = (unsigned char)((word >> (q - 1 - b)) & 1);
      ++n;
    }
  *Q = q;
  return n;
}

/* Threads an OpenMP region would use by default (1 without OpenMP). */
int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

static double clip(double v, double a) { return v < -a ? -a : (v > a ? a : v); }

/*
 * Whole path for every subcarrier: Algorithm 1, then Eq. 9.
 * mode 0 = MMSE (alpha = N0 / Es, projection = identity), 1 = BOX
 * (alpha = 0, projection of Eq. 14 with radius sqrt(Es) * max Re{O}).
 * llr may be NULL (then N0 may be 0).  threads <= 0: the OpenMP default.
 * Returns 0, or -1 for arguments outside the limits above.
 */
int orc_ocd_detect(const double* H, const double* Y, long long Nsc, int B, int U, int T,
                   double N0, double Es, int K, int mode, int order, double* z, double* llr,
                   int threads) {
  double pre[ORC_MAX_POINTS], pim[ORC_MAX_POINTS];
  unsigned char lab[ORC_MAX_POINTS][ORC_MAX_Q];
  int Q = 0;
  const int npts = alphabet(order, pre, pim, lab, &Q);
  if (npts == 0 || B < 1 || B > ORC_MAX_B || U < 1 || U > ORC_MAX_U || T < 1 || K < 0 ||
      Nsc < 0 || !(Es > 0.0) || N0 < 0.0 || (llr && !(N0 > 0.0)))
    return -1;
  const double alpha = mode == 0 ? N0 / Es : 0.0;
  /* box radius: the largest in-phase amplitude of O at energy Es (Section II-D) */
  double rad = 0.0;
  for (int i = 0; i < npts; ++i)
    if (pre[i] > rad) rad = pre[i];
  rad *= sqrt(Es);
  const int nt = threads > 0 ? threads : orc_max_threads();
  (void)nt;

#pragma omp parallel for schedule(dynamic, 8) num_threads(nt)
  for (long long w = 0; w < Nsc; ++w) {
    const double* h = H + 2 * (size_t)w * B * U;
    double n[ORC_MAX_U], dinv[ORC_MAX_U], p[ORC_MAX_U];
    /* preprocessing (Algorithm 1) */
    for (int u = 0; u < U; ++u) {
      double s = 0.0;
      for (int b = 0; b < B; ++b) {
        const double hr = h[2 * (b * U + u)], hi = h[2 * (b * U + u) + 1];
        s += hr * hr + hi * hi;
      }
      n[u] = s;
      const double den = s + alpha;
      dinv[u] = den > 0.0 ? 1.0 / den : 0.0;
      p[u] = dinv[u] * s;
    }
    for (int t = 0; t < T; ++t) {
      const double* y = Y + 2 * ((size_t)w * T + t) * B;
      double r[2 * ORC_MAX_B], zz[2 * ORC_MAX_U];
      for (int b = 0; b < 2 * B; ++b) r[b] = y[b];      /* r = y */
      for (int u = 0; u < 2 * U; ++u) zz[u] = 0.0;      /* z = 0 */
      for (int k = 0; k < K; ++k)
        for (int u = 0; u < U; ++u) {
          /* c = h_u^H r */
          double cr = 0.0, ci = 0.0;
          for (int b = 0; b < B; ++b) {
            const double hr = h[2 * (b * U + u)], hi = h[2 * (b * U + u) + 1];
            cr += hr * r[2 * b] + hi * r[2 * b + 1];
            ci += hr * r[2 * b + 1] - hi * r[2 * b];
          }
          /* z_u' = proj(d_u^-1 c + p_u z_u) */
          double wr = dinv[u] * cr + p[u] * zz[2 * u];
          double wi = dinv[u] * ci + p[u] * zz[2 * u + 1];
          if (mode == 1) {
            wr = clip(wr, rad);
            wi = order == 2 ? 0.0 : clip(wi, rad);
          }
          const double dr = wr - zz[2 * u], di = wi - zz[2 * u + 1];
          /* r <- r - h_u dz (Eq. 15) */
          for (int b = 0; b < B; ++b) {
            const double hr = h[2 * (b * U + u)], hi = h[2 * (b * U + u) + 1];
            r[2 * b] -= hr * dr - hi * di;
            r[2 * b + 1] -= hr * di + hi * dr;
          }
          zz[2 * u] = wr;
          zz[2 * u + 1] = wi;
        }
      double* zo = z + 2 * ((size_t)w * T + t) * U;
      for (int u = 0; u < 2 * U; ++u) zo[u] = zz[u];
      if (!llr) continue;
      /* Eq. 9 with mu~ = p_u, rho~ = ||h_u||^2 Es / N0 (Section III-C) */
      for (int u = 0; u < U; ++u) {
        double* L = llr + (((size_t)w * T + t) * U + u) * Q;
        if (!(p[u] > 0.0)) {
          for (int b = 0; b < Q; ++b) L[b] = 0.0;
          continue;
        }
        const double xr = zz[2 * u] / p[u] / sqrt(Es), xi = zz[2 * u + 1] / p[u] / sqrt(Es);
        const double rho = n[u] * Es / N0;
        for (int b = 0; b < Q; ++b) {
          double d0 = INFINITY, d1 = INFINITY;
          for (int i = 0; i < npts; ++i) {
            const double er = xr - pre[i], ei = xi - pim[i];
            const double d = er * er + ei * ei;
            if (lab[i][b]) { if (d < d1) d1 = d; }
            else if (d < d0) d0 = d;
          }
          L[b] = rho * (d0 - d1);
        }
      }
    }
  }
  return 0;
}
