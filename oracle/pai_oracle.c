/*
 * pai_oracle.c -- FP64 CPU oracle for planar / line-detector photoacoustic
 * Fourier reconstruction (Haltmeier, Scherzer, Zangerl, "A Reconstruction
 * Algorithm for Photoacoustic Imaging based on the Nonuniform FFT").
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, table or constant with the CUDA library and never calls it.
 *
 * What it computes: the paper's "direct Fourier reconstruction" (Sec. 4, the
 * first of the compared Fourier algorithms): Eq. (fft-1a) as a direct lateral
 * DFT, Eq. (fft-2) by direct summation at every node, the weight of
 * Eq. (fft-0) and the inverse DFT of Eq. (fft-1).  Nothing is approximated,
 * so this is the exact quantity that the NUFFT algorithm (Algorithm 2)
 * approximates.  No blocking, fusion or reordering beyond the separable
 * evaluation of the multi-dimensional uniform DFTs (their kernels factorise).
 *
 * General grid (d = 2 line detector, d = 3 planar detector):
 *   data    p[x][y][n] = p(x*dx, y*dy, n*dt),  n = 0..nt-1        (Eq. gd)
 *   image   f[x][y][q] ~ f(x*dx, y*dy, q*dz),  q = 0..nz-1        (Eq. fd)
 *   lateral frequencies kx in [-nx/2, nx/2), ky in [-ny/2, ny/2),
 *   depth frequency l in [-nz/2, nz/2); index k is stored at k mod n.
 *   Kx = 2 pi kx/(nx dx), Ky = 2 pi ky/(ny dy), Kz = 2 pi l/(nz dz),
 *   |K| = sqrt(Kx^2 + Ky^2 + Kz^2).
 *   node (time-index units):   nu = sign(l) * c * dt * nt * |K| / (2 pi)
 *   weight:                    W  = c * (dt/dz) * 2|Kz| / |K|,  W := 0 at l = 0
 * With unit sound speed, dx = dz = dt and nx = nz = nt = N this is the paper's
 * omega_{k,l} = sign(l) sqrt(k^2 + l^2) and weight 2|l|/omega (Eq. dft-2d,
 * Eq. fft-0).  The factor c*dt/dz follows from the exact inversion formula
 * Eq. (inv) after substituting tau = c t and discretising both Fourier
 * integrals with the trapezoid rule (Eq. dft-2d).
 *
 * Readings of the paper taken here (each is also listed in the design notes):
 *  - weight numerator is 2|Kz| (the depth frequency), as in Eq. (inv) and
 *    Eq. (inv2); the printed "2k" of Eq. (dft-2d)/(fft-0) uses the lateral
 *    index and is read as a typo;
 *  - sign(0) = 0 makes the l = 0 node 0 and the weight 0/0: the l = 0 entry of
 *    the image spectrum is set to 0 (the continuous limit of 2|Kz|/|K| at
 *    Kz -> 0 for Kx != 0);
 *  - Eq. (fft-1) is read as f_{m,n} = N^-2 sum_{k,l=-N/2}^{N/2-1}
 *    e^{+i(km+ln)2pi/N} fhat_{k,l} (m lateral, n depth), and the image is the
 *    real part of that sum (the l = -nz/2 row is not Hermitian-paired);
 *  - Algorithm 2 feeds row k of the lateral transform to the row NUFFT.
 *
 * Complex arrays are interleaved (re, im) doubles, i.e. C99 double _Complex,
 * the same memory layout as numpy complex128.
 */
#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

typedef double _Complex cplx;

typedef struct {
  int dim;          /* 2 (line detector) or 3 (planar detector)            */
  int nx, ny;       /* detector / lateral image grid; ny = 1 when dim == 2 */
  double dx, dy;    /* lateral spacings                                    */
  int nt;           /* time samples                                        */
  double dt;        /* time step                                           */
  double c;         /* sound speed                                         */
  int nz;           /* image depth samples                                 */
  double dz;        /* depth spacing                                       */
} oracle_geom;

/* ------------------------------------------------------------------ */
/* small helpers                                                       */
/* ------------------------------------------------------------------ */

static const double TWO_PI = 6.283185307179586476925286766559;

/* signed frequency of storage index i on an n-point grid */
static int signed_freq(int i, int n) { return (i < n / 2) ? i : i - n; }

/* e^{-2 pi i m / n} for m = 0..n-1, each entry from its own exact angle */
static cplx* twiddle_table(int n) {
  cplx* w = (cplx*)malloc(sizeof(cplx) * (size_t)n);
  if (!w) return NULL;
  for (int m = 0; m < n; ++m) {
    double a = TWO_PI * (double)m / (double)n;
    w[m] = cos(a) - I * sin(a);
  }
  return w;
}

static int n_threads(int requested) {
  if (requested > 0) return requested;
  long n = sysconf(_SC_NPROCESSORS_ONLN);
  return n > 0 ? (int)n : 1;
}

/* minimal parallel-for over [0, count): each worker takes a contiguous slice */
typedef void (*row_fn)(void* ctx, long row);
typedef struct { row_fn fn; void* ctx; long lo, hi; } slice_t;

static void* run_slice(void* a) {
  slice_t* s = (slice_t*)a;
  for (long r = s->lo; r < s->hi; ++r) s->fn(s->ctx, r);
  return NULL;
}

static void parallel_rows(row_fn fn, void* ctx, long count, int threads) {
  int t = n_threads(threads);
  if (t > count) t = (int)(count > 0 ? count : 1);
  if (t <= 1) {
    for (long r = 0; r < count; ++r) fn(ctx, r);
    return;
  }
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)t);
  slice_t* sl = (slice_t*)malloc(sizeof(slice_t) * (size_t)t);
  int started = 0;
  for (int i = 0; i < t; ++i) {
    sl[i].fn = fn; sl[i].ctx = ctx;
    sl[i].lo = count * i / t; sl[i].hi = count * (i + 1) / t;
    if (pthread_create(&th[i], NULL, run_slice, &sl[i]) == 0) started = i + 1;
    else { run_slice(&sl[i]); }
  }
  for (int i = 0; i < started; ++i) pthread_join(th[i], NULL);
  free(th); free(sl);
}

/* ------------------------------------------------------------------ */
/* nodes and weights (Eq. dft-2d nodes, Eq. fft-0 weight)              */
/* ------------------------------------------------------------------ */

/* |K| for signed frequencies (kx, ky, l) */
static double k_norm(const oracle_geom* g, int kx, int ky, int l) {
  double Kx = TWO_PI * kx / (g->nx * g->dx);
  double Ky = (g->dim == 3) ? TWO_PI * ky / (g->ny * g->dy) : 0.0;
  double Kz = TWO_PI * l / (g->nz * g->dz);
  return sqrt(Kx * Kx + Ky * Ky + Kz * Kz);
}

/* node nu_{k,l} in time-index units: the temporal DFT is evaluated at
 * omega = nu, i.e. sum_n e^{-i 2 pi nu n / nt} (Eq. fft-2) */
double oracle_node(const oracle_geom* g, int kx, int ky, int l) {
  double s = (l > 0) ? 1.0 : (l < 0 ? -1.0 : 0.0);
  return s * g->c * g->dt * g->nt * k_norm(g, kx, ky, l) / TWO_PI;
}

/* weight of Eq. (fft-0) in the general grid; 0 on the l = 0 row */
double oracle_weight(const oracle_geom* g, int kx, int ky, int l) {
  if (l == 0) return 0.0;
  double Kz = fabs(TWO_PI * l / (g->nz * g->dz));
  return g->c * (g->dt / g->dz) * 2.0 * Kz / k_norm(g, kx, ky, l);
}

/* all nodes and weights of one lateral row, storage index l mod nz */
void oracle_row_nodes(const oracle_geom* g, int kx, int ky, double* nu, double* w) {
  for (int li = 0; li < g->nz; ++li) {
    int l = signed_freq(li, g->nz);
    nu[li] = oracle_node(g, kx, ky, l);
    w[li] = oracle_weight(g, kx, ky, l);
  }
}

/* ------------------------------------------------------------------ */
/* Eq. (dft): direct DFT of one vector at arbitrary nodes               */
/* ------------------------------------------------------------------ */

/* out[i] = sum_{n=0}^{nt-1} e^{-i 2 pi nu_i n / nt} g[n]
 * Each angle is reduced to one turn in FP64 before cos/sin. */
void oracle_nudft(int nt, const cplx* g, int nnodes, const double* nu, cplx* out) {
  for (int i = 0; i < nnodes; ++i) {
    cplx acc = 0;
    for (int n = 0; n < nt; ++n) {
      double turns = nu[i] * (double)n / (double)nt;
      turns -= floor(turns);
      double a = TWO_PI * turns;
      acc += (cos(a) - I * sin(a)) * g[n];
    }
    out[i] = acc;
  }
}

/* adjoint of oracle_nudft: out[n] = sum_i e^{+i 2 pi nu_i n / nt} h[i] */
void oracle_nudft_adjoint(int nt, const cplx* h, int nnodes, const double* nu, cplx* out) {
  for (int n = 0; n < nt; ++n) {
    cplx acc = 0;
    for (int i = 0; i < nnodes; ++i) {
      double turns = nu[i] * (double)n / (double)nt;
      turns -= floor(turns);
      double a = TWO_PI * turns;
      acc += (cos(a) + I * sin(a)) * h[i];
    }
    out[n] = acc;
  }
}

/* ------------------------------------------------------------------ */
/* Step 1 -- Eq. (fft-1a): direct lateral DFT                          */
/* ------------------------------------------------------------------ */

typedef struct {
  const oracle_geom* g;
  const double* p;   /* real [nx][ny][nt] */
  cplx* tmp;         /* [kx][y][nt]        */
  cplx* pt;          /* [kx][ky][nt]       */
  const cplx* wx; const cplx* wy;
} lat_ctx;

/* along x: tmp[kx][y][n] = sum_x e^{-2 pi i kx x/nx} p[x][y][n] */
static void lat_x_row(void* a, long kx) {
  lat_ctx* c = (lat_ctx*)a;
  const oracle_geom* g = c->g;
  size_t plane = (size_t)g->ny * g->nt;
  cplx* dst = c->tmp + (size_t)kx * plane;
  for (size_t i = 0; i < plane; ++i) dst[i] = 0;
  for (int x = 0; x < g->nx; ++x) {
    cplx w = c->wx[((long)kx * x) % g->nx];
    const double* src = c->p + (size_t)x * plane;
    for (size_t i = 0; i < plane; ++i) dst[i] += w * src[i];
  }
}

/* along y: pt[kx][ky][n] = sum_y e^{-2 pi i ky y/ny} tmp[kx][y][n] */
static void lat_y_row(void* a, long kx) {
  lat_ctx* c = (lat_ctx*)a;
  const oracle_geom* g = c->g;
  size_t plane = (size_t)g->ny * g->nt;
  const cplx* src = c->tmp + (size_t)kx * plane;
  cplx* dst = c->pt + (size_t)kx * plane;
  for (int ky = 0; ky < g->ny; ++ky) {
    cplx* d = dst + (size_t)ky * g->nt;
    for (int n = 0; n < g->nt; ++n) d[n] = 0;
    for (int y = 0; y < g->ny; ++y) {
      cplx w = c->wy[((long)ky * y) % g->ny];
      const cplx* s = src + (size_t)y * g->nt;
      for (int n = 0; n < g->nt; ++n) d[n] += w * s[n];
    }
  }
}

/* pt[kx][ky][n] (complex) = lateral DFT of real p[x][y][n]; ny = 1 in 2-D */
int oracle_lateral_dft(const oracle_geom* g, const double* p, cplx* pt, int threads) {
  size_t total = (size_t)g->nx * g->ny * g->nt;
  lat_ctx c = {g, p, NULL, pt, NULL, NULL};
  c.tmp = (cplx*)malloc(sizeof(cplx) * total);
  c.wx = twiddle_table(g->nx);
  c.wy = twiddle_table(g->ny);
  if (!c.tmp || !c.wx || !c.wy) { free(c.tmp); free((void*)c.wx); free((void*)c.wy); return -1; }
  parallel_rows(lat_x_row, &c, g->nx, threads);
  parallel_rows(lat_y_row, &c, g->nx, threads);
  free(c.tmp); free((void*)c.wx); free((void*)c.wy);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Steps 2+3 -- Eq. (fft-2) by direct summation, weight Eq. (fft-0)    */
/* ------------------------------------------------------------------ */

typedef struct {
  const oracle_geom* g;
  const cplx* pt;    /* [kx][ky][nt] */
  cplx* fhat;        /* [kx][ky][nz] */
} spec_ctx;

static void spectrum_row(void* a, long row) {
  spec_ctx* c = (spec_ctx*)a;
  const oracle_geom* g = c->g;
  int kx = signed_freq((int)(row / g->ny), g->nx);
  int ky = signed_freq((int)(row % g->ny), g->ny);
  double* nu = (double*)malloc(sizeof(double) * (size_t)g->nz);
  cplx* P = (cplx*)malloc(sizeof(cplx) * (size_t)g->nz);
  for (int li = 0; li < g->nz; ++li) nu[li] = oracle_node(g, kx, ky, signed_freq(li, g->nz));
  oracle_nudft(g->nt, c->pt + (size_t)row * g->nt, g->nz, nu, P);
  cplx* dst = c->fhat + (size_t)row * g->nz;
  for (int li = 0; li < g->nz; ++li)
    dst[li] = oracle_weight(g, kx, ky, signed_freq(li, g->nz)) * P[li];
  free(nu); free(P);
}

/* image spectrum fhat[kx][ky][l] (all l, storage index l mod nz) */
int oracle_spectrum(const oracle_geom* g, const double* p, cplx* fhat, int threads) {
  size_t rows = (size_t)g->nx * g->ny;
  cplx* pt = (cplx*)malloc(sizeof(cplx) * rows * g->nt);
  if (!pt) return -1;
  if (oracle_lateral_dft(g, p, pt, threads)) { free(pt); return -1; }
  spec_ctx c = {g, pt, fhat};
  parallel_rows(spectrum_row, &c, (long)rows, threads);
  free(pt);
  return 0;
}

/* Selected rows only: for each requested signed lateral frequency pair
 * (kx[r], ky[r]) compute its lateral DFT row directly from p and then
 * fhat_r[l] for all l (storage index l mod nz).  Cost per row is
 * O(nx ny nt + nz nt), so large grids can be sampled row by row. */
typedef struct {
  const oracle_geom* g; const double* p; const int* kx; const int* ky; cplx* out;
} rows_ctx;

static void selected_row(void* a, long r) {
  rows_ctx* c = (rows_ctx*)a;
  const oracle_geom* g = c->g;
  int kx = c->kx[r], ky = c->ky[r];
  cplx* row = (cplx*)calloc((size_t)g->nt, sizeof(cplx));
  double* nu = (double*)malloc(sizeof(double) * (size_t)g->nz);
  for (int x = 0; x < g->nx; ++x)
    for (int y = 0; y < g->ny; ++y) {
      long mx = ((long)kx * x) % g->nx; if (mx < 0) mx += g->nx;
      long my = ((long)ky * y) % g->ny; if (my < 0) my += g->ny;
      double turns = (double)mx / g->nx + (double)my / g->ny;
      double ang = TWO_PI * turns;
      cplx w = cos(ang) - I * sin(ang);
      const double* src = c->p + ((size_t)x * g->ny + y) * g->nt;
      for (int n = 0; n < g->nt; ++n) row[n] += w * src[n];
    }
  for (int li = 0; li < g->nz; ++li) nu[li] = oracle_node(g, kx, ky, signed_freq(li, g->nz));
  cplx* dst = c->out + (size_t)r * g->nz;
  oracle_nudft(g->nt, row, g->nz, nu, dst);
  for (int li = 0; li < g->nz; ++li) dst[li] *= oracle_weight(g, kx, ky, signed_freq(li, g->nz));
  free(row); free(nu);
}

int oracle_spectrum_rows(const oracle_geom* g, const double* p, int nrows, const int* kx,
                         const int* ky, cplx* out, int threads) {
  rows_ctx c = {g, p, kx, ky, out};
  parallel_rows(selected_row, &c, nrows, threads);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Step 4 -- Eq. (fft-1): direct inverse DFT, real part                */
/* ------------------------------------------------------------------ */

typedef struct {
  const oracle_geom* g;
  const cplx* src; cplx* dst; double* out;
  const cplx* w; int sign;  /* w = e^{-2pi i m/n}; sign=+1 uses conj(w) */
} inv_ctx;

/* along depth, per lateral row: dst[row][q] = sum_l e^{+2 pi i l q/nz} src[row][l] */
static void inv_z_row(void* a, long row) {
  inv_ctx* c = (inv_ctx*)a;
  int nz = c->g->nz;
  const cplx* s = c->src + (size_t)row * nz;
  cplx* d = c->dst + (size_t)row * nz;
  for (int q = 0; q < nz; ++q) {
    cplx acc = 0;
    for (int li = 0; li < nz; ++li) {
      int l = signed_freq(li, nz);
      long m = ((long)l * q) % nz; if (m < 0) m += nz;
      acc += conj(c->w[m]) * s[li];
    }
    d[q] = acc;
  }
}

/* along x for fixed x-output: dst[x][y][q] = sum_kx e^{+2 pi i kx x/nx} src[kx][y][q] */
static void inv_x_row(void* a, long x) {
  inv_ctx* c = (inv_ctx*)a;
  const oracle_geom* g = c->g;
  size_t plane = (size_t)g->ny * g->nz;
  cplx* d = c->dst + (size_t)x * plane;
  for (size_t i = 0; i < plane; ++i) d[i] = 0;
  for (int ki = 0; ki < g->nx; ++ki) {
    int k = signed_freq(ki, g->nx);
    long m = ((long)k * x) % g->nx; if (m < 0) m += g->nx;
    cplx w = conj(c->w[m]);
    const cplx* s = c->src + (size_t)ki * plane;
    for (size_t i = 0; i < plane; ++i) d[i] += w * s[i];
  }
}

/* along y for fixed (x): dst[x][y][q] = sum_ky e^{+2 pi i ky y/ny} src[x][ky][q] */
static void inv_y_row(void* a, long x) {
  inv_ctx* c = (inv_ctx*)a;
  const oracle_geom* g = c->g;
  size_t plane = (size_t)g->ny * g->nz;
  const cplx* s = c->src + (size_t)x * plane;
  cplx* d = c->dst + (size_t)x * plane;
  for (int y = 0; y < g->ny; ++y) {
    cplx* dd = d + (size_t)y * g->nz;
    for (int q = 0; q < g->nz; ++q) dd[q] = 0;
    for (int ki = 0; ki < g->ny; ++ki) {
      int k = signed_freq(ki, g->ny);
      long m = ((long)k * y) % g->ny; if (m < 0) m += g->ny;
      cplx w = conj(c->w[m]);
      const cplx* ss = s + (size_t)ki * g->nz;
      for (int q = 0; q < g->nz; ++q) dd[q] += w * ss[q];
    }
  }
}

/* f[x][y][q] = Re( (nx ny nz)^-1 sum_{kx,ky,l} e^{+2 pi i(...)} fhat[kx][ky][l] ) */
int oracle_image_from_spectrum(const oracle_geom* g, const cplx* fhat, double* f, int threads) {
  size_t total = (size_t)g->nx * g->ny * g->nz;
  cplx* a = (cplx*)malloc(sizeof(cplx) * total);
  cplx* b = (cplx*)malloc(sizeof(cplx) * total);
  cplx* wz = twiddle_table(g->nz);
  cplx* wx = twiddle_table(g->nx);
  cplx* wy = twiddle_table(g->ny);
  if (!a || !b || !wz || !wx || !wy) { free(a); free(b); free(wz); free(wx); free(wy); return -1; }
  inv_ctx c = {g, fhat, a, NULL, wz, 1};
  parallel_rows(inv_z_row, &c, (long)g->nx * g->ny, threads);      /* a = IDFT_z */
  inv_ctx cx = {g, a, b, NULL, wx, 1};
  parallel_rows(inv_x_row, &cx, g->nx, threads);                   /* b = IDFT_x a */
  const cplx* res = b;
  if (g->dim == 3) {
    inv_ctx cy = {g, b, a, NULL, wy, 1};
    parallel_rows(inv_y_row, &cy, g->nx, threads);                 /* a = IDFT_y b */
    res = a;
  }
  double scale = 1.0 / ((double)g->nx * g->ny * g->nz);
  for (size_t i = 0; i < total; ++i) f[i] = creal(res[i]) * scale;
  free(a); free(b); free(wz); free(wx); free(wy);
  return 0;
}

/* The whole direct Fourier reconstruction: real p[x][y][n] -> real f[x][y][q] */
int oracle_reconstruct(const oracle_geom* g, const double* p, double* f, int threads) {
  size_t rows = (size_t)g->nx * g->ny;
  cplx* fhat = (cplx*)malloc(sizeof(cplx) * rows * g->nz);
  if (!fhat) return -1;
  int rc = oracle_spectrum(g, p, fhat, threads);
  if (!rc) rc = oracle_image_from_spectrum(g, fhat, f, threads);
  free(fhat);
  return rc;
}

/* ------------------------------------------------------------------ */
/* Adjoint: exact transpose of oracle_reconstruct under real inner      */
/* products.  With L = IDFT_d o diag(W) o NUDFT o DFT_lat (complex      */
/* linear) and the reconstruction f = Re(L p):                          */
/*   <Re(L p), h> = Re <L p, h> = <p, Re(L^H h)>  for real p, h,         */
/* so the adjoint is  p_bar = Re( DFT_lat^H NUDFT^H diag(W) IDFT_d^H h ),  */
/* with IDFT_d^H = (nx ny nz)^-1 * forward DFT (e^{-i}).                 */
/* ------------------------------------------------------------------ */

typedef struct {
  const oracle_geom* g; const cplx* F; cplx* pt;
} adj_ctx;

/* per lateral row: pt[row][n] = sum_l e^{+i 2 pi nu n/nt} W F[row][l] */
static void adjoint_row(void* a, long row) {
  adj_ctx* c = (adj_ctx*)a;
  const oracle_geom* g = c->g;
  int kx = signed_freq((int)(row / g->ny), g->nx);
  int ky = signed_freq((int)(row % g->ny), g->ny);
  double* nu = (double*)malloc(sizeof(double) * (size_t)g->nz);
  cplx* h = (cplx*)malloc(sizeof(cplx) * (size_t)g->nz);
  for (int li = 0; li < g->nz; ++li) {
    int l = signed_freq(li, g->nz);
    nu[li] = oracle_node(g, kx, ky, l);
    h[li] = oracle_weight(g, kx, ky, l) * c->F[(size_t)row * g->nz + li];
  }
  oracle_nudft_adjoint(g->nt, h, g->nz, nu, c->pt + (size_t)row * g->nt);
  free(nu); free(h);
}

/* forward DFT along depth: dst[row][l] = sum_q e^{-2 pi i l q/nz} src[row][q] */
typedef struct { const oracle_geom* g; const double* f; cplx* dst; const cplx* w; } fz_ctx;
static void fwd_z_row(void* a, long row) {
  fz_ctx* c = (fz_ctx*)a;
  int nz = c->g->nz;
  const double* s = c->f + (size_t)row * nz;
  cplx* d = c->dst + (size_t)row * nz;
  for (int li = 0; li < nz; ++li) {
    int l = signed_freq(li, nz);
    cplx acc = 0;
    for (int q = 0; q < nz; ++q) {
      long m = ((long)l * q) % nz; if (m < 0) m += nz;
      acc += c->w[m] * s[q];
    }
    d[li] = acc;
  }
}

/* forward DFT along x (per output kx) and along y (per x row), complex in place */
typedef struct { const oracle_geom* g; const cplx* src; cplx* dst; const cplx* w; int last; } fl_ctx;
static void fwd_x_row(void* a, long ki) {
  fl_ctx* c = (fl_ctx*)a;
  const oracle_geom* g = c->g;
  size_t plane = (size_t)g->ny * c->last;
  int k = signed_freq((int)ki, g->nx);
  cplx* d = c->dst + (size_t)ki * plane;
  for (size_t i = 0; i < plane; ++i) d[i] = 0;
  for (int x = 0; x < g->nx; ++x) {
    long m = ((long)k * x) % g->nx; if (m < 0) m += g->nx;
    const cplx* s = c->src + (size_t)x * plane;
    for (size_t i = 0; i < plane; ++i) d[i] += c->w[m] * s[i];
  }
}
static void fwd_y_row(void* a, long x) {
  fl_ctx* c = (fl_ctx*)a;
  const oracle_geom* g = c->g;
  size_t plane = (size_t)g->ny * c->last;
  const cplx* s = c->src + (size_t)x * plane;
  cplx* d = c->dst + (size_t)x * plane;
  for (int ki = 0; ki < g->ny; ++ki) {
    int k = signed_freq(ki, g->ny);
    cplx* dd = d + (size_t)ki * c->last;
    for (int q = 0; q < c->last; ++q) dd[q] = 0;
    for (int y = 0; y < g->ny; ++y) {
      long m = ((long)k * y) % g->ny; if (m < 0) m += g->ny;
      const cplx* ss = s + (size_t)y * c->last;
      for (int q = 0; q < c->last; ++q) dd[q] += c->w[m] * ss[q];
    }
  }
}

/* inverse-sign lateral sums for the adjoint: p_bar[x][y][n] =
 * Re sum_{kx,ky} e^{+2 pi i(kx x/nx + ky y/ny)} pt[kx][ky][n] */
typedef struct { const oracle_geom* g; const cplx* src; cplx* dst; const cplx* w; int last; } il_ctx;
static void adj_x_row(void* a, long x) {
  il_ctx* c = (il_ctx*)a;
  const oracle_geom* g = c->g;
  size_t plane = (size_t)g->ny * c->last;
  cplx* d = c->dst + (size_t)x * plane;
  for (size_t i = 0; i < plane; ++i) d[i] = 0;
  for (int ki = 0; ki < g->nx; ++ki) {
    int k = signed_freq(ki, g->nx);
    long m = ((long)k * x) % g->nx; if (m < 0) m += g->nx;
    cplx w = conj(c->w[m]);
    const cplx* s = c->src + (size_t)ki * plane;
    for (size_t i = 0; i < plane; ++i) d[i] += w * s[i];
  }
}
static void adj_y_row(void* a, long x) {
  il_ctx* c = (il_ctx*)a;
  const oracle_geom* g = c->g;
  size_t plane = (size_t)g->ny * c->last;
  const cplx* s = c->src + (size_t)x * plane;
  cplx* d = c->dst + (size_t)x * plane;
  for (int y = 0; y < g->ny; ++y) {
    cplx* dd = d + (size_t)y * c->last;
    for (int q = 0; q < c->last; ++q) dd[q] = 0;
    for (int ki = 0; ki < g->ny; ++ki) {
      int k = signed_freq(ki, g->ny);
      long m = ((long)k * y) % g->ny; if (m < 0) m += g->ny;
      cplx w = conj(c->w[m]);
      const cplx* ss = s + (size_t)ki * c->last;
      for (int q = 0; q < c->last; ++q) dd[q] += w * ss[q];
    }
  }
}

int oracle_adjoint(const oracle_geom* g, const double* h, double* pbar, int threads) {
  size_t rows = (size_t)g->nx * g->ny;
  size_t nimg = rows * g->nz, ndat = rows * g->nt;
  size_t nbig = nimg > ndat ? nimg : ndat;
  cplx* a = (cplx*)malloc(sizeof(cplx) * nbig);
  cplx* b = (cplx*)malloc(sizeof(cplx) * nbig);
  cplx* wz = twiddle_table(g->nz);
  cplx* wx = twiddle_table(g->nx);
  cplx* wy = twiddle_table(g->ny);
  if (!a || !b || !wz || !wx || !wy) { free(a); free(b); free(wz); free(wx); free(wy); return -1; }
  /* IDFT_d^H h = (nx ny nz)^-1 DFT_d h : depth, then x, then y */
  fz_ctx cz = {g, h, a, wz};
  parallel_rows(fwd_z_row, &cz, (long)rows, threads);
  fl_ctx cx = {g, a, b, wx, g->nz};
  parallel_rows(fwd_x_row, &cx, g->nx, threads);
  cplx* F = b;
  if (g->dim == 3) {
    fl_ctx cy = {g, b, a, wy, g->nz};
    parallel_rows(fwd_y_row, &cy, g->nx, threads);
    F = a;
  }
  double scale = 1.0 / ((double)g->nx * g->ny * g->nz);
  for (size_t i = 0; i < nimg; ++i) F[i] *= scale;
  /* NUDFT^H diag(W) per lateral row */
  cplx* pt = (F == a) ? b : a;
  adj_ctx ca = {g, F, pt};
  parallel_rows(adjoint_row, &ca, (long)rows, threads);
  /* DFT_lat^H and real part */
  cplx* o = (pt == a) ? b : a;
  il_ctx ix = {g, pt, o, wx, g->nt};
  parallel_rows(adj_x_row, &ix, g->nx, threads);
  const cplx* res = o;
  if (g->dim == 3) {
    il_ctx iy = {g, o, pt, wy, g->nt};
    parallel_rows(adj_y_row, &iy, g->nx, threads);
    res = pt;
  }
  for (size_t i = 0; i < ndat; ++i) pbar[i] = creal(res[i]);
  free(a); free(b); free(wz); free(wx); free(wy);
  return 0;
}

/* ------------------------------------------------------------------ */
/* The adjoint on a box of output samples (large grids)                */
/* ------------------------------------------------------------------ */

typedef struct {
  const oracle_geom* g; const cplx* F; cplx* q; int n0, cn;
} box_row_ctx;

/* q[row][n'] = sum_l e^{+i 2 pi nu (n0 + n') / nt} W F[row][l], n' < cn */
static void box_row(void* a, long row) {
  box_row_ctx* c = (box_row_ctx*)a;
  const oracle_geom* g = c->g;
  int kx = signed_freq((int)(row / g->ny), g->nx);
  int ky = signed_freq((int)(row % g->ny), g->ny);
  for (int j = 0; j < c->cn; ++j) c->q[(size_t)row * c->cn + j] = 0;
  for (int li = 0; li < g->nz; ++li) {
    int l = signed_freq(li, g->nz);
    double nu = oracle_node(g, kx, ky, l);
    cplx h = oracle_weight(g, kx, ky, l) * c->F[(size_t)row * g->nz + li];
    for (int j = 0; j < c->cn; ++j) {
      double turns = nu * (double)(c->n0 + j) / (double)g->nt;
      turns -= floor(turns);
      double ang = TWO_PI * turns;
      c->q[(size_t)row * c->cn + j] += (cos(ang) + I * sin(ang)) * h;
    }
  }
}

typedef struct {
  const oracle_geom* g; const cplx* q; const cplx* wx; const cplx* wy;
  int x0, y0, cy, cn; double* out;
} box_lat_ctx;

/* out[x'][y'][n'] = Re sum_{kx,ky} e^{+2 pi i (kx x/nx + ky y/ny)} q[kx][ky][n'] */
static void box_lat(void* a, long xi) {
  box_lat_ctx* c = (box_lat_ctx*)a;
  const oracle_geom* g = c->g;
  int x = c->x0 + (int)xi;
  cplx* acc = (cplx*)calloc((size_t)c->cy * c->cn, sizeof(cplx));
  for (int ki = 0; ki < g->nx; ++ki) {
    int kx = signed_freq(ki, g->nx);
    long mx = ((long)kx * x) % g->nx; if (mx < 0) mx += g->nx;
    cplx wxv = conj(c->wx[mx]);
    for (int kj = 0; kj < g->ny; ++kj) {
      int ky = signed_freq(kj, g->ny);
      const cplx* src = c->q + ((size_t)ki * g->ny + kj) * c->cn;
      for (int yi = 0; yi < c->cy; ++yi) {
        int y = c->y0 + yi;
        long my = ((long)ky * y) % g->ny; if (my < 0) my += g->ny;
        cplx w = wxv * conj(c->wy[my]);
        cplx* d = acc + (size_t)yi * c->cn;
        for (int j = 0; j < c->cn; ++j) d[j] += w * src[j];
      }
    }
  }
  for (size_t i = 0; i < (size_t)c->cy * c->cn; ++i) c->out[(size_t)xi * c->cy * c->cn + i] = creal(acc[i]);
  free(acc);
}

/* The adjoint of oracle_reconstruct restricted to the output box
 * x in [x0, x0+cx), y in [y0, y0+cy) (y0 = 0, cy = 1 in 2-D), n in [n0, n0+cn):
 * out[x'][y'][n'] = pbar[x0+x'][y0+y'][n0+n'] with the same sums as
 * oracle_adjoint (image-side DFT in full, the temporal and lateral adjoint sums
 * only at the requested samples). */
int oracle_adjoint_box(const oracle_geom* g, const double* h, int x0, int cx, int y0, int cy, int n0, int cn,
                       double* out, int threads) {
  if (x0 < 0 || cx < 1 || x0 + cx > g->nx || y0 < 0 || cy < 1 || y0 + cy > g->ny || n0 < 0 || cn < 1 ||
      n0 + cn > g->nt)
    return -2;
  size_t rows = (size_t)g->nx * g->ny;
  size_t nimg = rows * g->nz;
  cplx* a = (cplx*)malloc(sizeof(cplx) * nimg);
  cplx* b = (cplx*)malloc(sizeof(cplx) * nimg);
  cplx* q = (cplx*)malloc(sizeof(cplx) * rows * (size_t)cn);
  cplx* wz = twiddle_table(g->nz);
  cplx* wx = twiddle_table(g->nx);
  cplx* wy = twiddle_table(g->ny);
  if (!a || !b || !q || !wz || !wx || !wy) {
    free(a); free(b); free(q); free(wz); free(wx); free(wy);
    return -1;
  }
  fz_ctx cz = {g, h, a, wz};
  parallel_rows(fwd_z_row, &cz, (long)rows, threads);
  fl_ctx cxx = {g, a, b, wx, g->nz};
  parallel_rows(fwd_x_row, &cxx, g->nx, threads);
  cplx* F = b;
  if (g->dim == 3) {
    fl_ctx cy_ = {g, b, a, wy, g->nz};
    parallel_rows(fwd_y_row, &cy_, g->nx, threads);
    F = a;
  }
  double scale = 1.0 / ((double)g->nx * g->ny * g->nz);
  for (size_t i = 0; i < nimg; ++i) F[i] *= scale;
  box_row_ctx cr = {g, F, q, n0, cn};
  parallel_rows(box_row, &cr, (long)rows, threads);
  box_lat_ctx cl = {g, q, wx, wy, x0, y0, cy, cn, out};
  parallel_rows(box_lat, &cl, cx, threads);
  free(a); free(b); free(q); free(wz); free(wx); free(wy);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Discrete forward model (the operator Q of Sec. 2 on a padded box)    */
/* ------------------------------------------------------------------ */
/*
 * The image f[x][y][q] sits at the origin of a periodic box of bx x by x bz
 * cells (zeros elsewhere).  The wave equation with initial pressure equal to
 * the box's trigonometric interpolant and zero initial velocity has the
 * solution  sum_K fhat(K) cos(c |K| t) e^{i K.r} / (bx by bz);  at the
 * detectors (depth 0, lateral cells x < nx, y < ny) and times t_n = n dt:
 *   p[x][y][n] = Re (1/(bx by bz)) sum_{kx,ky,l} fhat[kx][ky][l]
 *                cos(2 pi nu n / nt) e^{+2 pi i (kx x/bx + ky y/by)},
 *   nu = c dt nt |K| / (2 pi),  K = 2 pi (kx/(bx dx), ky/(by dy), l/(bz dz)),
 * signed frequencies, fhat the unnormalised DFT of the padded image.
 */
typedef struct {
  const oracle_geom* g; int bx, by, bz;
  const double* f; cplx* A; cplx* B; cplx* C; const cplx* wx; const cplx* wy; const cplx* wz;
  double* out;
} fm_ctx;

/* A[kx][y][q] = sum_{x < nx} e^{-2 pi i kx x / bx} f[x][y][q] */
static void fm_x(void* a, long kx) {
  fm_ctx* c = (fm_ctx*)a;
  const oracle_geom* g = c->g;
  size_t plane = (size_t)g->ny * g->nz;
  cplx* d = c->A + (size_t)kx * plane;
  for (size_t i = 0; i < plane; ++i) d[i] = 0;
  for (int x = 0; x < g->nx; ++x) {
    cplx w = c->wx[((long)kx * x) % c->bx];
    const double* s = c->f + (size_t)x * plane;
    for (size_t i = 0; i < plane; ++i) d[i] += w * s[i];
  }
}

/* B[kx][ky][q] = sum_{y < ny} e^{-2 pi i ky y / by} A[kx][y][q] */
static void fm_y(void* a, long kx) {
  fm_ctx* c = (fm_ctx*)a;
  const oracle_geom* g = c->g;
  const cplx* s = c->A + (size_t)kx * g->ny * g->nz;
  cplx* d = c->B + (size_t)kx * c->by * g->nz;
  for (int ky = 0; ky < c->by; ++ky) {
    cplx* dd = d + (size_t)ky * g->nz;
    for (int q = 0; q < g->nz; ++q) dd[q] = 0;
    for (int y = 0; y < g->ny; ++y) {
      cplx w = c->wy[((long)ky * y) % c->by];
      const cplx* ss = s + (size_t)y * g->nz;
      for (int q = 0; q < g->nz; ++q) dd[q] += w * ss[q];
    }
  }
}

/* C[kx][ky][n] = (1/(bx by bz)) sum_l cos(2 pi nu n/nt) sum_{q < nz} e^{-2 pi i l q/bz} B[kx][ky][q] */
static void fm_t(void* a, long kx) {
  fm_ctx* c = (fm_ctx*)a;
  const oracle_geom* g = c->g;
  int skx = signed_freq((int)kx, c->bx);
  cplx* F = (cplx*)malloc(sizeof(cplx) * (size_t)c->bz);
  double scale = 1.0 / ((double)c->bx * c->by * c->bz);
  for (int ky = 0; ky < c->by; ++ky) {
    int sky = signed_freq(ky, c->by);
    const cplx* s = c->B + ((size_t)kx * c->by + ky) * g->nz;
    for (int l = 0; l < c->bz; ++l) {
      cplx acc = 0;
      for (int q = 0; q < g->nz; ++q) acc += c->wz[((long)l * q) % c->bz] * s[q];
      F[l] = acc;
    }
    cplx* d = c->C + ((size_t)kx * c->by + ky) * g->nt;
    for (int n = 0; n < g->nt; ++n) d[n] = 0;
    for (int l = 0; l < c->bz; ++l) {
      int sl = signed_freq(l, c->bz);
      double Kx = TWO_PI * skx / (c->bx * g->dx);
      double Ky = (g->dim == 3) ? TWO_PI * sky / (c->by * g->dy) : 0.0;
      double Kz = TWO_PI * sl / (c->bz * g->dz);
      double nu = g->c * g->dt * g->nt * sqrt(Kx * Kx + Ky * Ky + Kz * Kz) / TWO_PI;
      for (int n = 0; n < g->nt; ++n) {
        double turns = nu * (double)n / (double)g->nt;
        turns -= floor(turns);
        d[n] += cos(TWO_PI * turns) * F[l];
      }
    }
    for (int n = 0; n < g->nt; ++n) d[n] *= scale;
  }
  free(F);
}

/* out[x][y][n] = Re sum_{kx,ky} e^{+2 pi i (kx x/bx + ky y/by)} C[kx][ky][n], x < nx, y < ny */
static void fm_lat(void* a, long x) {
  fm_ctx* c = (fm_ctx*)a;
  const oracle_geom* g = c->g;
  cplx* acc = (cplx*)calloc((size_t)g->ny * g->nt, sizeof(cplx));
  for (int kx = 0; kx < c->bx; ++kx) {
    cplx wxv = conj(c->wx[((long)kx * x) % c->bx]);
    for (int ky = 0; ky < c->by; ++ky) {
      const cplx* s = c->C + ((size_t)kx * c->by + ky) * g->nt;
      for (int y = 0; y < g->ny; ++y) {
        cplx w = wxv * conj(c->wy[((long)ky * y) % c->by]);
        cplx* d = acc + (size_t)y * g->nt;
        for (int n = 0; n < g->nt; ++n) d[n] += w * s[n];
      }
    }
  }
  for (size_t i = 0; i < (size_t)g->ny * g->nt; ++i) c->out[(size_t)x * g->ny * g->nt + i] = creal(acc[i]);
  free(acc);
}

int oracle_forward_model(const oracle_geom* g, const double* f, int bx, int by, int bz, double* p, int threads) {
  if (bx < g->nx || bz < g->nz || (g->dim == 3 && by < g->ny) || bx < 1 || bz < 1) return -2;
  if (g->dim != 3) by = 1;
  fm_ctx c;
  c.g = g; c.bx = bx; c.by = by; c.bz = bz; c.f = f; c.out = p;
  c.A = (cplx*)malloc(sizeof(cplx) * (size_t)bx * g->ny * g->nz);
  c.B = (cplx*)malloc(sizeof(cplx) * (size_t)bx * by * g->nz);
  c.C = (cplx*)malloc(sizeof(cplx) * (size_t)bx * by * g->nt);
  cplx* wx = twiddle_table(bx);
  cplx* wy = twiddle_table(by);
  cplx* wz = twiddle_table(bz);
  c.wx = wx; c.wy = wy; c.wz = wz;
  if (!c.A || !c.B || !c.C || !wx || !wy || !wz) {
    free(c.A); free(c.B); free(c.C); free(wx); free(wy); free(wz);
    return -1;
  }
  parallel_rows(fm_x, &c, bx, threads);
  parallel_rows(fm_y, &c, bx, threads);
  parallel_rows(fm_t, &c, bx, threads);
  parallel_rows(fm_lat, &c, g->nx, threads);
  free(c.A); free(c.B); free(c.C); free(wx); free(wy); free(wz);
  return 0;
}

int oracle_threads(int requested) { return n_threads(requested); }
