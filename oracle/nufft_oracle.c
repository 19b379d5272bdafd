/*
 * CPU oracle for the type-1 / type-2 NUFFT of Barnett, Magland & af Klinteberg,
 * "A parallel non-uniform fast Fourier transform library based on an
 * 'exponential of semicircle' kernel" (arXiv:1808.06736).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls
 * this file; only the test suite, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header or table with the CUDA library.
 *
 * Everything is IEEE double precision.  Complex arrays are interleaved
 * (re, im) pairs.  Point coordinates come as separate x, y, z arrays.
 *
 * Two levels (the Python wrapper in oracle/__init__.py drives both):
 *   O1  direct evaluation of the exponential sums, Eq. (1) and Eq. (2);
 *   O2  the plain ES-kernel algorithm of Sec. 3.1 / 3.2: spreading (Eq. (bl)),
 *       interpolation (Eq. (interp)) written as direct loops over points and
 *       kernel nodes.  The FFT and the diagonal correction steps are done in
 *       Python with numpy/scipy.
 *
 * Mode ordering of every mode array: increasing k in each dimension
 * (k_i from -floor(N_i/2)), dimension 1 fastest.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Kahan-compensated running sum of one real component. */
typedef struct { double s, e; } ksum;
static inline void kadd(ksum* a, double v) {
  double y = v - a->e;
  double t = a->s + y;
  a->e = (t - a->s) - y;
  a->s = t;
}

static const double* coord(int i, const double* x, const double* y, const double* z) {
  return i == 0 ? x : (i == 1 ? y : z);
}

/*
 * O1, type 1, Eq. (1):  f_k = sum_j c_j exp(i * isign * k.x_j)
 * evaluated for an explicit list of nk mode vectors k (nk x d integers,
 * row-major).  Used in full (all of I_N) for small problems and on a random
 * subset of modes for large ones.
 *
 * Threads split the modes when there are many, otherwise they split the
 * points (each thread sums a contiguous chunk; chunks are then added in
 * thread order).
 */
void oracle_type1_direct(int d, int64_t M, const double* x, const double* y, const double* z,
                         const double* c, int isign, int64_t nk, const int64_t* k, double* f) {
  int nthr = 1;
#ifdef _OPENMP
  nthr = omp_get_max_threads();
#endif
  if (nk >= 4 * nthr || M < 4096) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < nk; ++q) {
      ksum re = {0, 0}, im = {0, 0};
      for (int64_t j = 0; j < M; ++j) {
        double ph = 0;
        for (int i = 0; i < d; ++i) ph += (double)k[q * d + i] * coord(i, x, y, z)[j];
        ph *= (double)isign;
        double cs = cos(ph), sn = sin(ph);
        kadd(&re, c[2 * j] * cs - c[2 * j + 1] * sn);
        kadd(&im, c[2 * j] * sn + c[2 * j + 1] * cs);
      }
      f[2 * q] = re.s;
      f[2 * q + 1] = im.s;
    }
    return;
  }
  /* few modes, many points: split the points */
  double* part = (double*)calloc((size_t)nthr * (size_t)nk * 2, sizeof(double));
#pragma omp parallel
  {
    int t = 0, nt = 1;
#ifdef _OPENMP
    t = omp_get_thread_num();
    nt = omp_get_num_threads();
#endif
    int64_t j0 = M * t / nt, j1 = M * (t + 1) / nt;
    for (int64_t q = 0; q < nk; ++q) {
      ksum re = {0, 0}, im = {0, 0};
      for (int64_t j = j0; j < j1; ++j) {
        double ph = 0;
        for (int i = 0; i < d; ++i) ph += (double)k[q * d + i] * coord(i, x, y, z)[j];
        ph *= (double)isign;
        double cs = cos(ph), sn = sin(ph);
        kadd(&re, c[2 * j] * cs - c[2 * j + 1] * sn);
        kadd(&im, c[2 * j] * sn + c[2 * j + 1] * cs);
      }
      part[((size_t)t * nk + q) * 2] = re.s;
      part[((size_t)t * nk + q) * 2 + 1] = im.s;
    }
  }
  for (int64_t q = 0; q < nk; ++q) {
    ksum re = {0, 0}, im = {0, 0};
    for (int t = 0; t < nthr; ++t) {
      kadd(&re, part[((size_t)t * nk + q) * 2]);
      kadd(&im, part[((size_t)t * nk + q) * 2 + 1]);
    }
    f[2 * q] = re.s;
    f[2 * q + 1] = im.s;
  }
  free(part);
}

/*
 * O1, type 2, Eq. (2) with the sign flag of the interface:
 *   c_j = sum_{k in I_N} f_k exp(i * isign * k.x_j)
 * for nt target points (xt, yt, zt).  N[0..d-1] are the mode counts; f is in
 * the mode ordering stated in the file header.  exp(i isign k.x) is formed as
 * the product over dimensions of exp(i isign k_i x_i), each factor from one
 * cos/sin call.  The modes are summed in chunks of 4096 (Kahan inside a chunk,
 * chunks added in order), threads splitting the chunks.
 */
void oracle_type2_direct(int d, int64_t nt, const double* xt, const double* yt, const double* zt,
                         const int64_t* N, const double* f, int isign, double* c) {
  int64_t Nt = 1, Ni[3] = {1, 1, 1};
  for (int i = 0; i < d; ++i) { Ni[i] = N[i]; Nt *= N[i]; }
  const int64_t CH = 4096;
  int64_t nch = (Nt + CH - 1) / CH;
  double* e[3];
  for (int i = 0; i < 3; ++i) e[i] = (double*)malloc(sizeof(double) * 2 * (size_t)Ni[i]);
  double* part = (double*)malloc(sizeof(double) * 2 * (size_t)nch);
  for (int64_t j = 0; j < nt; ++j) {
    for (int i = 0; i < 3; ++i) {
      for (int64_t m = 0; m < Ni[i]; ++m) {
        if (i >= d) { e[i][2 * m] = 1.0; e[i][2 * m + 1] = 0.0; continue; }
        double kk = (double)(m - Ni[i] / 2);
        double ph = (double)isign * kk * coord(i, xt, yt, zt)[j];
        e[i][2 * m] = cos(ph);
        e[i][2 * m + 1] = sin(ph);
      }
    }
#pragma omp parallel for schedule(static)
    for (int64_t ch = 0; ch < nch; ++ch) {
      ksum re = {0, 0}, im = {0, 0};
      int64_t m1 = (ch + 1) * CH < Nt ? (ch + 1) * CH : Nt;
      for (int64_t m = ch * CH; m < m1; ++m) {
        int64_t a = m % Ni[0], b = (m / Ni[0]) % Ni[1], q = m / (Ni[0] * Ni[1]);
        /* e1*e2*e3 */
        double pr = e[0][2 * a] * e[1][2 * b] - e[0][2 * a + 1] * e[1][2 * b + 1];
        double pi = e[0][2 * a] * e[1][2 * b + 1] + e[0][2 * a + 1] * e[1][2 * b];
        double er = pr * e[2][2 * q] - pi * e[2][2 * q + 1];
        double ei = pr * e[2][2 * q + 1] + pi * e[2][2 * q];
        kadd(&re, f[2 * m] * er - f[2 * m + 1] * ei);
        kadd(&im, f[2 * m] * ei + f[2 * m + 1] * er);
      }
      part[2 * ch] = re.s;
      part[2 * ch + 1] = im.s;
    }
    ksum re = {0, 0}, im = {0, 0};
    for (int64_t ch = 0; ch < nch; ++ch) { kadd(&re, part[2 * ch]); kadd(&im, part[2 * ch + 1]); }
    c[2 * j] = re.s;
    c[2 * j + 1] = im.s;
  }
  for (int i = 0; i < 3; ++i) free(e[i]);
  free(part);
}

/*
 * kernel = 0: the ES kernel, Eq. (ES): phi(z) = exp(beta (sqrt(1 - z^2) - 1)).
 * kernel = 1: its smooth variant of the Remark in Sec. 7,
 *   phi(z) = 2 exp(-beta) cosh(beta sqrt(1 - z^2)),
 * a power series in 1 - z^2, so smooth up to z = +-1, and within exp(-beta) of ES.
 * Both are zero for |z| > 1.
 */
static double es_kernel(double z, double beta, int kernel) {
  if (fabs(z) > 1.0) return 0.0;
  if (kernel == 1) return 2.0 * exp(-beta) * cosh(beta * sqrt(1.0 - z * z));
  return exp(beta * (sqrt(1.0 - z * z) - 1.0));
}

/*
 * The w grid nodes one coordinate touches, with their kernel values, for the
 * periodised rescaled kernel of Eqs. (al), (psi1), (ppsi1):
 *   psi~(l h - x) = sum_m phi((l h - x - 2 pi m) / alpha),  alpha = w h / 2,
 *   h = 2 pi / n.
 * With u = x / h the argument is (l - u) * 2 / w.  The nodes taken are the w
 * consecutive integers starting at ceil(u - w/2) (the kernel's support holds
 * w + 1 nodes only when u - w/2 is an integer, where the extra node has
 * weight exp(-beta)).  Each node is reported by its index modulo n, which is
 * how the periodisation acts on the grid since n >= 2w.
 */
static void node_weights(double x, int64_t n, int w, double beta, int kernel, int64_t* idx, double* ker) {
  const double two_pi = 6.283185307179586476925286766559;
  double u = x * (double)n / two_pi;
  double l0 = ceil(u - 0.5 * (double)w);
  for (int t = 0; t < w; ++t) {
    double l = l0 + (double)t;
    ker[t] = es_kernel((l - u) * 2.0 / (double)w, beta, kernel);
    int64_t li = (int64_t)l % n;
    if (li < 0) li += n;
    idx[t] = li;
  }
}

/*
 * O2 step 1 of type 1, Eq. (bl) (1D form Eq. (bl1)):
 *   b_l = sum_j c_j psi~(l_1 h_1 - x_j, ..., l_d h_d - z_j)
 * with the tensor-product kernel of Eq. (ppsi).  b (n_1 x ... x n_d complex,
 * dimension 1 fastest) is overwritten.  A plain loop over points, then over
 * the w^d nodes of each point.
 *
 * Threads own slabs of the last dimension's grid index (no atomics): every
 * thread walks all points in order and adds only the nodes whose last index
 * lies in its slab.  Each grid value therefore receives its contributions in
 * point order, exactly as a single thread would add them.
 */
void oracle_spread(int d, int64_t M, const double* x, const double* y, const double* z,
                   const double* c, const int64_t* n, int w, double beta, int kernel, double* b) {
  int64_t nn[3] = {1, 1, 1}, nt = 1;
  for (int i = 0; i < d; ++i) { nn[i] = n[i]; nt *= n[i]; }
  memset(b, 0, sizeof(double) * 2 * (size_t)nt);
  const int last = d - 1;
  const int64_t nl = nn[last];
  const double two_pi = 6.283185307179586476925286766559;
#pragma omp parallel
  {
    int th = 0, nth = 1;
#ifdef _OPENMP
    th = omp_get_thread_num();
    nth = omp_get_num_threads();
#endif
    const int64_t lo = nl * th / nth, hi = nl * (th + 1) / nth; /* this thread's slab [lo, hi) */
    int64_t idx[3][32];
    double ker[3][32];
    const int wd[3] = {w, d >= 2 ? w : 1, d >= 3 ? w : 1};
    for (int64_t j = 0; j < M && lo < hi; ++j) {
      /* skip points none of whose last-dimension nodes lies in the slab */
      double u = coord(last, x, y, z)[j] * (double)nl / two_pi;
      int64_t s0 = (int64_t)ceil(u - 0.5 * (double)w) % nl;
      if (s0 < 0) s0 += nl;
      int touches = 0;
      for (int t = 0; t < w && !touches; ++t) {
        int64_t li = (s0 + t) % nl;
        touches = li >= lo && li < hi;
      }
      if (!touches) continue;
      for (int i = 0; i < 3; ++i) {
        if (i < d) node_weights(coord(i, x, y, z)[j], nn[i], w, beta, kernel, idx[i], ker[i]);
        else { idx[i][0] = 0; ker[i][0] = 1.0; }
      }
      for (int t3 = 0; t3 < wd[2]; ++t3)
        for (int t2 = 0; t2 < wd[1]; ++t2)
          for (int t1 = 0; t1 < w; ++t1) {
            const int tl = last == 0 ? t1 : (last == 1 ? t2 : t3);
            if (idx[last][tl] < lo || idx[last][tl] >= hi) continue;
            double kv = ker[0][t1] * ker[1][t2] * ker[2][t3];
            int64_t g = idx[0][t1] + nn[0] * (idx[1][t2] + nn[1] * idx[2][t3]);
            b[2 * g] += c[2 * j] * kv;
            b[2 * g + 1] += c[2 * j + 1] * kv;
          }
    }
  }
}

/*
 * O2 step 3 of type 2, Eq. (interp):
 *   c_j = sum_l b_l psi~(l_1 h_1 - x_j, ..., l_d h_d - z_j)
 * over the same w^d nodes as oracle_spread, which makes it the exact
 * transpose of that spreading map.
 */
void oracle_interp(int d, int64_t M, const double* x, const double* y, const double* z,
                   const double* b, const int64_t* n, int w, double beta, int kernel, double* c) {
  int64_t nn[3] = {1, 1, 1};
  for (int i = 0; i < d; ++i) nn[i] = n[i];
  /* points are independent: threads split them */
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < M; ++j) {
    int64_t idx[3][32];
    double ker[3][32];
    int w2 = d >= 2 ? w : 1, w3 = d >= 3 ? w : 1;
    for (int i = 0; i < 3; ++i) {
      if (i < d) node_weights(coord(i, x, y, z)[j], nn[i], w, beta, kernel, idx[i], ker[i]);
      else { idx[i][0] = 0; ker[i][0] = 1.0; }
    }
    double sr = 0, si = 0;
    for (int t3 = 0; t3 < w3; ++t3)
      for (int t2 = 0; t2 < w2; ++t2)
        for (int t1 = 0; t1 < w; ++t1) {
          double kv = ker[0][t1] * ker[1][t2] * ker[2][t3];
          int64_t g = idx[0][t1] + nn[0] * (idx[1][t2] + nn[1] * idx[2][t3]);
          sr += b[2 * g] * kv;
          si += b[2 * g + 1] * kv;
        }
    c[2 * j] = sr;
    c[2 * j + 1] = si;
  }
}

/*
 * Eq. (3), the type-3 sum: f_k = sum_j c_j exp(i isign s_k . x_j) for nt
 * real target frequencies (s, t, u = their coordinates), Kahan sums over the
 * sources, threads over the targets.
 */
void oracle_type3_direct(int d, int64_t M, const double* x, const double* y, const double* z, const double* c,
                         int isign, int64_t nt, const double* s, const double* t, const double* u, double* f) {
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t q = 0; q < nt; ++q) {
    ksum re = {0, 0}, im = {0, 0};
    for (int64_t j = 0; j < M; ++j) {
      double ph = 0;
      for (int i = 0; i < d; ++i) ph += coord(i, s, t, u)[q] * coord(i, x, y, z)[j];
      ph *= (double)isign;
      double cs = cos(ph), sn = sin(ph);
      kadd(&re, c[2 * j] * cs - c[2 * j + 1] * sn);
      kadd(&im, c[2 * j] * sn + c[2 * j + 1] * cs);
    }
    f[2 * q] = re.s;
    f[2 * q + 1] = im.s;
  }
}

/* Number of OpenMP threads the direct sums, spreading and interpolation use (1 without OpenMP). */
int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Set that number (n >= 1); returns the number now in effect. */
int oracle_set_num_threads(int n) {
#ifdef _OPENMP
  if (n >= 1) omp_set_num_threads(n);
#endif
  return oracle_num_threads();
}
