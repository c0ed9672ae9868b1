/*
 * FP64 CPU oracle for the tcFFT method (arXiv 2104.11471).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into liboracle.so, which
 * only the test suite, the package's smoke check and the benchmark's CPU
 * baseline load.  The GPU library never links or calls it, and it shares no
 * code, header, table or constant with the GPU path.
 *
 * What it computes (all forward, sign -, unnormalised, complex double,
 * interleaved re/im):
 *   oracle_dft_brute   -- the DFT definition, Eq. (dft_def) of Sec. 2.1:
 *                         X[k] = sum_n x[n] exp(-2 pi i n k / N), O(N^2).
 *   oracle_dft_bins    -- the same definition evaluated for selected k only
 *                         (used to check full-size GPU results bin by bin).
 *   oracle_fft_radix2  -- Cooley-Tukey with N1 = 2 applied recursively:
 *                         the merge of Eq. (dft_s2), X[k] = sum_m W_N^{mk}
 *                         X_m[k mod N2], with x_m[n] = x[n N1 + m].
 *   oracle_fft_mixed   -- the same recursion with caller-chosen radices, each
 *                         merge written as the matrix form of Eq. (dft_mm):
 *                         X_out = F_{N1} . (T_{N1 N2} (.) X_in).
 *   oracle_merge       -- one merging process of Eq. (dft_mm) on its own.
 *   oracle_fft_batch   -- batched 1D transforms (radix-2), threads over batch.
 *   oracle_fft_2d      -- batched 2D transforms on row-major [nx][ny] data:
 *                         ny-point transforms of the rows, then nx-point
 *                         transforms of the columns (Sec. 3.1, "Support
 *                         batched FFT and 2D FFT").
 *
 * Twiddles W_N^a = exp(-2 pi i a / N) are formed with exact integer argument
 * reduction: a is reduced mod N, folded to the first octant by the symmetries
 * of sine and cosine, and only then passed to libm sin/cos.  This keeps the
 * twiddle error at ~1 ulp for every N up to 2^30.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  double re, im;
} cplx;

static inline cplx cmul(cplx a, cplx b) {
  cplx r = {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
  return r;
}
static inline cplx cadd(cplx a, cplx b) {
  cplx r = {a.re + b.re, a.im + b.im};
  return r;
}
static inline cplx csub(cplx a, cplx b) {
  cplx r = {a.re - b.re, a.im - b.im};
  return r;
}

/* W_N^a = exp(-2 pi i a / N) for integer a, N > 0. */
static cplx twiddle(int64_t a, int64_t n) {
  int64_t r = a % n;
  if (r < 0) r += n;
  /* The angle 2 pi r / n is split with integer arithmetic into an octant
   * index q and an exact remainder: 8 r = q n + s, 0 <= s < n, so the angle
   * is (q + s/n) pi/4.  Even octants are evaluated from t = (s/n) pi/4,
   * odd octants from the complement u = pi/4 - t = ((n-s)/n) pi/4, so libm
   * only ever sees an argument in [0, pi/4]. */
  int64_t q = (8 * r) / n;
  int64_t s = 8 * r - q * n;
  double cr, sr; /* cos and sin of the angle */
  if ((q & 1) == 0) {
    double t = (double)s / (double)n * (M_PI / 4.0);
    double c = cos(t), sn = sin(t);
    switch (q) {
      case 0: cr = c; sr = sn; break;    /* t */
      case 2: cr = -sn; sr = c; break;   /* pi/2 + t */
      case 4: cr = -c; sr = -sn; break;  /* pi + t */
      default: cr = sn; sr = -c; break;  /* 3pi/2 + t */
    }
  } else {
    double u = (double)(n - s) / (double)n * (M_PI / 4.0);
    double cu = cos(u), su = sin(u);
    switch (q) {
      case 1: cr = su; sr = cu; break;   /* pi/2 - u */
      case 3: cr = -cu; sr = su; break;  /* pi - u */
      case 5: cr = -su; sr = -cu; break; /* 3pi/2 - u */
      default: cr = cu; sr = -su; break; /* 2pi - u */
    }
  }
#if defined(ORACLE_PLANT) && ORACLE_PLANT == 1
  cplx w = {cr, sr}; /* planted: wrong sign of the exponent */
#else
  cplx w = {cr, -sr};
#endif
  return w;
}

/* ------------------------------------------------------------- Eq. dft_def */
void oracle_dft_brute(int64_t n, const double* in, double* out) {
  const cplx* x = (const cplx*)in;
  cplx* X = (cplx*)out;
  for (int64_t k = 0; k < n; ++k) {
    cplx acc = {0.0, 0.0};
    for (int64_t j = 0; j < n; ++j) acc = cadd(acc, cmul(x[j], twiddle(j * k % n, n)));
    X[k] = acc;
  }
}

typedef struct {
  int64_t n, nbins;
  const cplx* x;
  const int64_t* bins;
  cplx* out;
  int64_t lo, hi;
} bins_job;

static void* bins_worker(void* arg) {
  bins_job* jb = (bins_job*)arg;
  for (int64_t b = jb->lo; b < jb->hi; ++b) {
    int64_t k = jb->bins[b] % jb->n;
    cplx acc = {0.0, 0.0};
    /* exponent j*k mod n accumulated incrementally to stay exact */
    int64_t e = 0;
    for (int64_t j = 0; j < jb->n; ++j) {
      acc = cadd(acc, cmul(jb->x[j], twiddle(e, jb->n)));
      e += k;
      if (e >= jb->n) e -= jb->n;
    }
    jb->out[b] = acc;
  }
  return NULL;
}

/* X[bins[i]] of one transform by the definition, threads over bins. */
void oracle_dft_bins(int64_t n, const double* in, int64_t nbins, const int64_t* bins,
                     double* out, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > nbins) nthreads = (int)(nbins > 0 ? nbins : 1);
  pthread_t th[256];
  bins_job jobs[256];
  if (nthreads > 256) nthreads = 256;
  for (int t = 0; t < nthreads; ++t) {
    jobs[t].n = n;
    jobs[t].nbins = nbins;
    jobs[t].x = (const cplx*)in;
    jobs[t].bins = bins;
    jobs[t].out = (cplx*)out;
    jobs[t].lo = nbins * t / nthreads;
    jobs[t].hi = nbins * (t + 1) / nthreads;
    pthread_create(&th[t], NULL, bins_worker, &jobs[t]);
  }
  for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
}

/* ------------------------------------------------------ Eq. dft_s2, N1 = 2 */
/* Out-of-place recursion: the sub-sequences x_m[n] = x[2n + m] (m = 0, 1)
 * are transformed into out[0 .. n/2) and out[n/2 .. n), then merged with
 * X[k] = X_0[k] + W_n^k X_1[k], X[k + n/2] = X_0[k] - W_n^k X_1[k].
 * tw holds W_ntop^j for j < ntop/2; W_n^k = W_ntop^{k * ntop / n}. */
static void r2_rec(const cplx* x, int64_t stride, int64_t n, cplx* out, const cplx* tw,
                   int64_t ntop) {
  if (n == 1) {
    out[0] = x[0];
    return;
  }
  int64_t h = n / 2;
  r2_rec(x, 2 * stride, h, out, tw, ntop);
  r2_rec(x + stride, 2 * stride, h, out + h, tw, ntop);
  int64_t step = ntop / n;
  for (int64_t k = 0; k < h; ++k) {
    cplx e = out[k];
#if defined(ORACLE_PLANT) && ORACLE_PLANT == 3
    cplx o = cmul(tw[(k * step + step) % (ntop / 2 > 0 ? ntop / 2 : 1)], out[k + h]); /* planted: twiddle index off by one */
#elif defined(ORACLE_PLANT) && ORACLE_PLANT == 6
    /* planted: in the last merge, the twiddle of one thin output slice
     * (k = 3 mod ntop/16) is taken ntop/8 entries too far */
    int64_t ti = (n == ntop && ntop >= 64 && k % (ntop / 16) == 3) ? (k * step + ntop / 8) % (ntop / 2) : k * step;
    cplx o = cmul(tw[ti], out[k + h]);
#else
    cplx o = cmul(tw[k * step], out[k + h]);
#endif
    out[k] = cadd(e, o);
    out[k + h] = csub(e, o);
  }
}

static cplx* r2_table(int64_t n) {
  int64_t h = n / 2 > 0 ? n / 2 : 1;
  cplx* tw = (cplx*)malloc(sizeof(cplx) * (size_t)h);
  for (int64_t j = 0; j < h; ++j) tw[j] = twiddle(j, n);
  return tw;
}

/* one transform, n a power of two */
void oracle_fft_radix2(int64_t n, const double* in, double* out) {
  cplx* tw = r2_table(n);
  r2_rec((const cplx*)in, 1, n, (cplx*)out, tw, n);
  free(tw);
}

/* ------------------------------------------------------------ Eq. dft_mm */
/* One merging process.  xin is the N1 x N2 matrix X_in (row m = X_m, the
 * N2-point DFT of the m-th decimated sub-sequence); xout is the N1 x N2
 * matrix X_out whose row l holds X[l N2 .. l N2 + N2).  With N = N1 N2,
 *   X_out[l][k2] = sum_m F_{N1}[l][m] * (T[m][k2] * X_in[m][k2]),
 *   F_{N1}[l][m] = W_{N1}^{l m},  T[m][k2] = W_N^{m k2}. */
void oracle_merge(int64_t n1, int64_t n2, const double* xin, double* xout) {
  const cplx* Xi = (const cplx*)xin;
  cplx* Xo = (cplx*)xout;
  int64_t n = n1 * n2;
  cplx* y = (cplx*)malloc(sizeof(cplx) * (size_t)n);
  for (int64_t m = 0; m < n1; ++m) /* element-wise product T (.) X_in */
    for (int64_t k2 = 0; k2 < n2; ++k2)
#if defined(ORACLE_PLANT) && ORACLE_PLANT == 2
      y[m * n2 + k2] = Xi[m * n2 + k2]; /* planted: twiddle T dropped */
#else
      y[m * n2 + k2] = cmul(twiddle(m * k2, n), Xi[m * n2 + k2]);
#endif
  for (int64_t l = 0; l < n1; ++l) /* matrix product F . (T (.) X_in) */
    for (int64_t k2 = 0; k2 < n2; ++k2) {
      cplx acc = {0.0, 0.0};
      for (int64_t m = 0; m < n1; ++m)
#if defined(ORACLE_PLANT) && ORACLE_PLANT == 4
        acc = cadd(acc, cmul(twiddle(l * m, n1), y[l * n2 + k2])); /* planted: F operand index transposed */
#else
        acc = cadd(acc, cmul(twiddle(l * m, n1), y[m * n2 + k2]));
#endif
      Xo[l * n2 + k2] = acc;
    }
  free(y);
}

/* Recursive mixed-radix: radices[0] = N1 is the outermost merge. The
 * product of radices must equal n (a radix list of length 0 means n == 1). */
static void mixed_rec(const cplx* x, int64_t stride, int64_t n, const int64_t* radices,
                      int nr, cplx* out) {
  if (n == 1) {
    out[0] = x[0];
    return;
  }
  int64_t n1 = radices[0], n2 = n / n1;
  cplx* xin = (cplx*)malloc(sizeof(cplx) * (size_t)n);
  for (int64_t m = 0; m < n1; ++m) /* X_m = DFT of x_m[j] = x[j N1 + m] */
    mixed_rec(x + m * stride, stride * n1, n2, radices + 1, nr - 1, xin + m * n2);
  oracle_merge(n1, n2, (const double*)xin, (double*)out);
  free(xin);
}

/* returns 0 on success, -1 if the radices do not multiply to n */
int oracle_fft_mixed(int64_t n, const int64_t* radices, int nr, const double* in, double* out) {
  int64_t p = 1;
  for (int i = 0; i < nr; ++i) p *= radices[i];
  if (p != n) return -1;
  mixed_rec((const cplx*)in, 1, n, radices, nr, (cplx*)out);
  return 0;
}

/* ------------------------------------------------------------- batched 1D */
typedef struct {
  int64_t n, lo, hi;
  const cplx* in;
  cplx* out;
  const cplx* tw;
} batch_job;

static void* batch_worker(void* arg) {
  batch_job* jb = (batch_job*)arg;
  for (int64_t b = jb->lo; b < jb->hi; ++b)
    r2_rec(jb->in + b * jb->n, 1, jb->n, jb->out + b * jb->n, jb->tw, jb->n);
  return NULL;
}

void oracle_fft_batch(int64_t n, int64_t batch, const double* in, double* out, int nthreads) {
  cplx* tw = r2_table(n);
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  if (nthreads > batch) nthreads = (int)(batch > 0 ? batch : 1);
  pthread_t th[256];
  batch_job jobs[256];
  for (int t = 0; t < nthreads; ++t) {
    jobs[t].n = n;
    jobs[t].lo = batch * t / nthreads;
    jobs[t].hi = batch * (t + 1) / nthreads;
    jobs[t].in = (const cplx*)in;
    jobs[t].out = (cplx*)out;
    jobs[t].tw = tw;
    pthread_create(&th[t], NULL, batch_worker, &jobs[t]);
  }
  for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
  free(tw);
}

/* ------------------------------------------------------------- batched 2D */
typedef struct {
  int64_t nx, ny, lo, hi; /* work items: rows or columns of all batches */
  int pass;               /* 0 rows, 1 columns */
  const cplx* in;
  cplx* out;
  const cplx* tw;
} td_job;

static void* td_worker(void* arg) {
  td_job* jb = (td_job*)arg;
  int64_t nx = jb->nx, ny = jb->ny;
  if (jb->pass == 0) {
    for (int64_t r = jb->lo; r < jb->hi; ++r) /* r = b * nx + ix */
      r2_rec(jb->in + r * ny, 1, ny, jb->out + r * ny, jb->tw, ny);
  } else {
    cplx* col = (cplx*)malloc(sizeof(cplx) * (size_t)nx);
    for (int64_t c = jb->lo; c < jb->hi; ++c) { /* c = b * ny + iy */
      int64_t b = c / ny, iy = c % ny;
      cplx* base = jb->out + b * nx * ny + iy;
#if defined(ORACLE_PLANT) && ORACLE_PLANT == 5
      r2_rec(base, 1, nx, col, jb->tw, nx); /* planted: column stride lost */
#else
      r2_rec(base, ny, nx, col, jb->tw, nx);
#endif
      for (int64_t ix = 0; ix < nx; ++ix) base[ix * ny] = col[ix];
    }
    free(col);
  }
  return NULL;
}

static void td_run(td_job* proto, int64_t items, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  if (nthreads > items) nthreads = (int)(items > 0 ? items : 1);
  pthread_t th[256];
  td_job jobs[256];
  for (int t = 0; t < nthreads; ++t) {
    jobs[t] = *proto;
    jobs[t].lo = items * t / nthreads;
    jobs[t].hi = items * (t + 1) / nthreads;
    pthread_create(&th[t], NULL, td_worker, &jobs[t]);
  }
  for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
}

/* data layout [batch][nx][ny], ny contiguous; out may not alias in */
void oracle_fft_2d(int64_t nx, int64_t ny, int64_t batch, const double* in, double* out,
                   int nthreads) {
  cplx* twy = r2_table(ny);
  cplx* twx = r2_table(nx);
  td_job p;
  p.nx = nx;
  p.ny = ny;
  p.in = (const cplx*)in;
  p.out = (cplx*)out;
  p.pass = 0;
  p.tw = twy;
  td_run(&p, batch * nx, nthreads);
  p.pass = 1;
  p.tw = twx;
  td_run(&p, batch * ny, nthreads);
  free(twy);
  free(twx);
}

/* exposed for tests of the twiddle generator itself */
void oracle_twiddle(int64_t a, int64_t n, double* out2) {
  cplx w = twiddle(a, n);
  out2[0] = w.re;
  out2[1] = w.im;
}
