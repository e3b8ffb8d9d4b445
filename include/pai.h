/*
 * pai.h -- C ABI of the GB300 (sm_103a) photoacoustic Fourier reconstruction
 * library (libpai.so).
 *
 * Method: Haltmeier, Scherzer, Zangerl, "A Reconstruction Algorithm for
 * Photoacoustic Imaging based on the Nonuniform FFT", Algorithm 2
 * ("FouRecNufft"), generalised from the paper's 2-D unit grid to line (d = 2)
 * and planar (d = 3) detectors on arbitrary rectangular grids:
 *
 *   1. lateral FFT of the detector data over the detector coordinate(s)
 *      (Eq. fft-1a);
 *   2. for every lateral frequency K_lat a 1-D nonuniform FFT along time
 *      (Algorithm 1: Kaiser-Bessel prescale, zero padding to the oversampled
 *      length c*nt, FFT, truncated window-weighted gather) evaluating the
 *      temporal spectrum at the nodes omega = c_s * sign(Kz) * |K|
 *      (Eq. fft-2, Eq. dft-2d);
 *   3. the weight of the exact inversion formula, 2|Kz|/|K| times
 *      c_s*dt/dz (Eq. fft-0, Eq. inv);
 *   4. the inverse FFT to the image, real part (Eq. fft-1).
 *
 * Grids.  Detector data p[x][y][n] = p(x*dx, y*dy, n*dt), n = 0..nt-1, t = 0
 * at the illumination.  Image f[x][y][q] ~ f(x*dx, y*dy, q*dz), q = 0..nz-1,
 * depth 0 = detector plane.  In 2-D drop the y index (ny = 1).  Both arrays
 * are FP32, contiguous, last index fastest.
 *
 * Memory.  Every pointer passed to pai_reconstruct / pai_adjoint is a DEVICE
 * pointer on the plan's device, owned by the caller, not retained after the
 * call.  Every pointer passed to pai_reconstruct_host is a HOST pointer.  The
 * plan owns its workspace, its cuFFT plans and its CUDA graphs.
 *
 * Streams.  All calls except pai_plan*, pai_destroy and pai_reconstruct_host
 * are asynchronous on the plan's stream (set at plan time, changeable with
 * pai_set_stream).  A plan must not be used by two host threads at once.
 *
 * Errors.  Every function returns a pai_status; nothing else crosses the ABI.
 * On failure, out-parameters are left untouched and no work is enqueued.
 */
#ifndef PAI_H
#define PAI_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pai_plan_s* pai_plan_t;

typedef enum {
  PAI_OK = 0,
  PAI_ERR_INVALID_ARG = 1,  /* bad geometry, size or pointer                 */
  PAI_ERR_UNSUPPORTED = 2,  /* valid but outside what this build implements  */
  PAI_ERR_OOM = 3,          /* device or host allocation failed              */
  PAI_ERR_CUDA = 4,         /* a CUDA runtime call or kernel launch failed   */
  PAI_ERR_CUFFT = 5,        /* a cuFFT call failed                           */
  PAI_ERR_TIMEOUT = 6       /* a bounded device-side wait gave up            */
} pai_status;

/* Problem statement (paper Sec. 2 and Sec. 4, Eq. gd / Eq. fd).
 * Parameters of the nonuniform FFT (Algorithm 1): 0 selects the default.   */
typedef struct {
  int dim;              /* 2 = line detector, 3 = planar detector             */
  int nx, ny;           /* detector grid = lateral image grid; ny = 1 in 2-D   */
  double dx, dy;        /* detector spacings (> 0)                            */
  int nt;               /* time samples (even, >= 2)                          */
  double dt;            /* time step (> 0)                                    */
  double c;             /* speed of sound (> 0)                               */
  int nz;               /* image depth samples (even, >= 2)                   */
  double dz;            /* depth spacing (> 0)                                */
  double oversampling;  /* NUFFT oversampling c_os > 1; 0 -> 2.  The padded
                           temporal FFT length is the smallest power of two
                           >= c_os*nt, so the effective c_os may be larger.  */
  double K;             /* interpolation length K (> 0); 0 -> chosen so the
                           window's truncation error is <= 1e-8.  The number of
                           taps per node is 2*ceil(c_os*K) and stays fixed when
                           the effective oversampling grows.                  */
  double alpha;         /* Kaiser-Bessel shape; 0 -> pi*(2c_os - 1)*(1 - 1e-3),
                           must be < pi*(2c_os - 1) (Lemma on Fourmont's
                           identity).                                        */
  int method;           /* how the temporal spectrum is evaluated at the nodes
                           (paper Sec. 4, the compared Fourier algorithms):
                           PAI_METHOD_KB (0, default): Algorithm 1 with the
                             Kaiser-Bessel window;
                           PAI_METHOD_TSINC: Algorithm 1 with the indicator
                             window of [-c pi, c pi] (truncated sinc, taps
                             2 ceil(c K), K default 3);
                           PAI_METHOD_LINEAR / PAI_METHOD_NEAREST: the exact
                             oversampled DFT at omega = j/c (no window),
                             interpolated linearly / to the nearest node;
                             oversampling may be 1 (no oversampling).
                           All problems of a batch use the same method.      */
} pai_geometry;

#define PAI_METHOD_KB 0
#define PAI_METHOD_TSINC 1
#define PAI_METHOD_LINEAR 2
#define PAI_METHOD_NEAREST 3

/* Read-only description of a plan (for reports and tests). */
typedef struct {
  int count;              /* problems in the plan (1 unless batched)            */
  int M;                  /* padded temporal FFT length of problem 0            */
  int taps;               /* grid values read per node: 2*ceil(c_os*K) for the
                             windowed methods, 2 (linear), 1 (nearest)          */
  double oversampling;    /* effective c_os = M/nt of problem 0                  */
  double K, alpha;        /* effective window parameters of problem 0 (alpha is
                             0 and K the tap half-width for the truncated sinc;
                             both 0 for the interpolation methods)             */
  double predicted_error; /* FP64 truncation error of the window identity (max
                             over the batch), see pai_plan; -1 for the
                             interpolation methods, which have no such bound     */
  int threads_per_cta;    /* row-kernel CTA size chosen by the tuner             */
  int ctas;               /* row-kernel grid size (persistent CTAs)              */
  int rows;               /* lateral-frequency rows processed per call          */
  long long nodes;        /* nodes evaluated per call (sum over the batch)      */
  size_t workspace_bytes; /* device bytes owned by the plan                     */
  int uses_graph;         /* 1 if calls replay a captured CUDA graph            */
  int library_ffts;       /* bit 0: pai_reconstruct runs every stage on the
                             library's own kernels (power-of-two sizes, chosen
                             by the tuner), else its inverse uses cuFFT; bit 1:
                             the same for pai_adjoint                          */
} pai_plan_info;

/* Create a plan for one reconstruction problem (Algorithm 2).
 * g:           problem statement; read during the call only.
 * cuda_stream: cudaStream_t (may be NULL = legacy default stream) on the
 *              current device; all later work of the plan is enqueued there.
 * out:         receives the plan on success.
 * Synchronises the device.  Validation (PAI_ERR_INVALID_ARG): dim in {2,3};
 * nx, nz, nt even and >= 2 (ny even and >= 2 in 3-D); spacings, dt and c > 0;
 * oversampling == 0 or > 1 (== 1 also allowed for PAI_METHOD_LINEAR and
 * PAI_METHOD_NEAREST); K >= 0; 0 <= alpha < pi*(2 c_os_eff - 1); method in
 * PAI_METHOD_KB..PAI_METHOD_NEAREST.                                         */
pai_status pai_plan(const pai_geometry* g, void* cuda_stream, pai_plan_t* out);

/* Create one plan for `count` independent 2-D or 3-D problems (g[0..count-1])
 * executed together: one lateral FFT per problem, ONE persistent row-kernel
 * launch over every lateral-frequency row of every problem, one inverse FFT
 * per problem, all replayed as one CUDA graph.  The problems share the tap
 * count and the method (PAI_ERR_INVALID_ARG otherwise); each keeps its own
 * oversampling.  When every problem leaves the window open (method KB, K,
 * oversampling and alpha all 0) the plan times window candidates -- for each
 * half tap count H, every problem's smallest power-of-two padded length whose
 * truncation error stays within 1e-7 and whose prescale spans at most a
 * factor 32 (low oversampling with many taps magnifies FP32 rounding) -- and
 * keeps the fastest (see
 * pai_tuning_log, pai_get_problem_info); otherwise the tap count is the
 * largest the problems ask for.
 * Data and images of the batch are concatenated in g-order.                  */
pai_status pai_plan_batched(const pai_geometry* g, int count, void* cuda_stream, pai_plan_t* out);

/* Reconstruction f = R p (Algorithm 2).
 * d_p: device, FP32, sum over problems of nx*ny*nt values, read only.
 * d_f: device, FP32, sum over problems of nx*ny*nz values, overwritten.
 * Both start on an 8-byte boundary (the kernels move two floats at a time;
 * PAI_ERR_INVALID_ARG otherwise, as for pai_adjoint and pai_spectrum).
 * Asynchronous on the plan's stream.                                         */
pai_status pai_reconstruct(pai_plan_t plan, const float* d_p, float* d_f);

/* Adjoint p_bar = R^T h of the operator pai_reconstruct applies (the exact
 * transpose of the discretised Algorithm 2 under real inner products:
 * forward image FFT, window spread from the nodes onto the oversampled grid
 * in gather form, inverse oversampled FFT, prescale, inverse lateral FFT).
 * d_h: device, FP32, image-shaped, read only.  d_pbar: device, FP32,
 * data-shaped, overwritten; both 8-byte aligned.  Asynchronous on the plan's
 * stream.  For the
 * interpolation methods the transposed interpolation spreads each node onto
 * its one or two grid cells, whose phases follow the spread.                 */
pai_status pai_adjoint(pai_plan_t plan, const float* d_h, float* d_pbar);

/* The image spectrum before the inverse FFT: steps 1-3 of Algorithm 2.
 * d_fhat: device, interleaved complex64, [nx][ny][nz/2+1] per problem
 * (half spectrum in depth, full lateral spectrum), including the factor
 * 1/(nx*ny*nz) of the inverse FFT.  Entry l = nz/2 holds the mean of the two
 * Nyquist nodes (the real part of the inverse DFT depends only on it).        */
pai_status pai_spectrum(pai_plan_t plan, const float* d_p, float* d_fhat);

/* End-to-end reconstruction from HOST memory: copies h_p to the device,
 * runs pai_reconstruct and copies the image back into h_f, then synchronises
 * the plan's stream.  h_p / h_f: host FP32 arrays sized as for
 * pai_reconstruct (page-locked memory gives full copy speed).  Uses
 * plan-owned device staging buffers allocated on first use.                  */
pai_status pai_reconstruct_host(pai_plan_t plan, const float* h_p, float* h_f);

/* The same, pipelined across calls (a stream of reconstructions from host
 * memory, e.g. successive frames): returns once the work is enqueued.  The
 * copy of this call's h_p to the device, its reconstruction and the copy of
 * its image into h_f run on three streams with two plan-owned device staging
 * pairs (allocated on first use), so one call's upload overlaps the previous
 * call's transforms and the download of the one before.  h_p and h_f must be
 * page-locked for the copies to be asynchronous (pageable memory still works,
 * but its copies block the caller).  The caller must not modify h_p nor read
 * h_f until pai_host_wait returns.  Not a paper operation: a transfer
 * schedule around pai_reconstruct.                                           */
pai_status pai_reconstruct_host_async(pai_plan_t plan, const float* h_p, float* h_f);

/* Block until every pai_reconstruct_host_async call on the plan has finished
 * (images in their h_f).                                                     */
pai_status pai_host_wait(pai_plan_t plan);

/* Per-stage device times for profiling.  Runs `reps` eager (not graph)
 * passes of pai_reconstruct (adjoint = 0) or pai_adjoint (adjoint = 1) on the
 * given device buffers with CUDA events between the stages, synchronises the
 * plan's stream and writes the mean milliseconds per pass of
 *   ms[0] the first cuFFT stage (lateral R2C; adjoint: image R2C),
 *   ms[1] the row kernel (forward: prescale + oversampled FFT + window gather
 *         + weight; adjoint: spread + inverse oversampled FFT + prescale),
 *   ms[2] the last cuFFT stage (image C2R; adjoint: lateral C2R).
 * d_in / d_out as for pai_reconstruct / pai_adjoint; ms: host, 3 doubles.   */
pai_status pai_profile_stages(pai_plan_t plan, const float* d_in, float* d_out, int reps, int adjoint, double* ms);

/* Change the stream later calls are enqueued on (cudaStream_t or NULL).     */
pai_status pai_set_stream(pai_plan_t plan, void* cuda_stream);

/* Spread of pai_adjoint and pai_forward_model (the transpose of the window
 * gather, Algorithm 1 read backwards).  Five spreads exist:
 *   atomic        shared-memory atomic adds per node (every node adds its 2H
 *                 tap contributions to the oversampled grid at once);
 *   runs          the same per run (the first node of each run of nodes on
 *                 the same grid cell sums the run and adds once per tap);
 *   tap           tap phases (nodes add tap by tap in a fixed order, one
 *                 barrier per phase);
 *   pairs         the nodes +-nu of a row as pairs, spread by one warp per row
 *                 (32 pairs at a time, runs summed by warp shuffles, plain
 *                 read-modify-writes; windowed methods, rows of 32 or 64
 *                 threads);
 *   pairs_atomic  the same by every warp of the row, adding with shared-memory
 *                 atomics (windowed methods).
 * tap and pairs are bit-identical on repeated calls; for the three atomic
 * spreads the order of the additions into one grid cell, hence the last bits
 * of the result, may differ from call to call.  pai_plan times every spread
 * that applies and keeps the fastest (the environment variable PAI_SPREAD
 * forces one by the names above).
 * deterministic = 1: the faster of tap and pairs; deterministic = 0: back to
 * the plan's choice.  pai_reconstruct is deterministic either way.  Waits for
 * the plan's stream and drops the plan's captured CUDA graphs (they are
 * captured again on next use).  Any other value: PAI_ERR_INVALID_ARG.      */
pai_status pai_set_deterministic(pai_plan_t plan, int deterministic);

/* Fill *info with the plan's parameters (M, oversampling, K and alpha of
 * problem 0; pai_get_problem_info gives them for every problem of a batch).  */
pai_status pai_get_info(pai_plan_t plan, pai_plan_info* info);

/* The window and padded length one problem of a plan runs with (Algorithm 1
 * parameters: c = M / nt, K = H / c with 2H taps, alpha = beta c).          */
typedef struct {
  int M;                  /* padded length of the oversampled temporal FFT      */
  int taps;               /* window taps per node (2H; 2 linear, 1 nearest)     */
  double oversampling;    /* c = M / nt                                        */
  double K;               /* half interpolation length in omega units, H / c    */
  double alpha;           /* Kaiser-Bessel shape (0 for other methods)          */
  double predicted_error; /* truncation error of Fourmont's identity (-1: none) */
} pai_problem_info;
/* index: 0 <= index < pai_plan_info.count, else PAI_ERR_INVALID_ARG.        */
pai_status pai_get_problem_info(pai_plan_t plan, int index, pai_problem_info* info);

/* What the plan's tuner measured when the plan was built and what it kept:
 * one line per measurement (window candidates: half tap count and padded
 * lengths with the forward row kernel's time; CTA sizes; adjoint spread
 * schemes; transform pipelines).  Copies at most cap - 1 bytes and a
 * terminating NUL into buf (buf may be NULL when cap is 0); *len (may be
 * NULL) receives the full length without the NUL.  Empty when the plan was
 * built without tuning.                                                      */
pai_status pai_tuning_log(pai_plan_t plan, char* buf, size_t cap, size_t* len);

/* Cumulative count of kernels and cuFFT executions this plan has enqueued
 * (graph replays count the kernels inside the graph).                        */
pai_status pai_launch_count(pai_plan_t plan, long long* kernels);

/* Release the plan and everything it owns.  Synchronises the plan's stream.
 * NULL is accepted and ignored.                                              */
pai_status pai_destroy(pai_plan_t plan);

/* Host-only probe of the plan-time window math (no GPU needed).  For half
 * tap count H = c*K, shape beta = alpha/c and oversampling c it writes
 * phi_out[i] = psi_hat(y_i / c) / psi_hat(0) for the n grid offsets y[i]
 * (the Kaiser-Bessel transform of Sec. 3.2 in grid units, analytic
 * continuation beyond |y| = H), and *pred_err = the largest error of
 * Fourmont's identity (Lemma in Sec. 3.1) truncated to the 2H taps, over
 * theta in [-pi, pi] and all node offsets, and *fit_err = the largest error
 * of the FP32 tap polynomials the kernels use, relative to psi_hat(0).
 * Any output pointer may be NULL.  Returns PAI_ERR_INVALID_ARG unless
 * 2 <= H <= 12, c > 1 and pi < beta*c <= pi*(2c - 1) (the paper's own example
 * alpha = 3 pi at c = 2 sits on that boundary).                              */
pai_status pai_window_probe(int H, double beta, double c, int n, const double* y, double* phi_out,
                            double* pred_err, double* fit_err);

/* Discrete forward model: the detector data of an initial pressure (the
 * operator Q of Sec. 2: the wave equation's solution on the detector plane,
 * depth 0, at the recorded times), for iterative or regularised
 * reconstruction around pai_reconstruct / pai_adjoint.
 *
 * Definition.  The image f[x][y][q] (the image grid of g) is zero-padded to a
 * periodic box of bx x by x bz cells, each extent the next power of two >= the
 * image extent + ceil(c nt dt / spacing) + 2 (so no periodic image of the
 * object reaches the detectors within the recorded time); the data are the
 * exact wave-equation solution for the trigonometric interpolant of the
 * padded image, p(x, t_n) = Re (1/(bx by bz)) sum_K fhat_box(K) cos(c |K| t_n)
 * e^{i K_lat x}, at the detector positions x < nx (y < ny).  Per lateral box
 * frequency the sum over depth frequencies is a cosine sum at the
 * nonuniform frequencies c|K|: a type-1 NUFFT (nodes +-nu, the Kaiser-Bessel
 * window of the plan parameters), evaluated by the adjoint pipeline on the
 * box.
 *
 * pai_forward_plan: g as for pai_plan (method KB or TSINC); box extents up to
 * 16384 laterally and 8192 in depth (PAI_ERR_UNSUPPORTED beyond); allocates
 * the box buffers (4 (bx by bz + bx by nt) bytes) besides the plan's own.
 * The returned plan accepts pai_forward_model, pai_forward_box, pai_get_info
 * (describing the box geometry), pai_set_stream, pai_launch_count,
 * pai_profile_stages with adjoint = 1 (box-sized buffers) and pai_destroy;
 * the other calls return PAI_ERR_INVALID_ARG.
 * pai_forward_model: d_f device FP32 image [nx][ny][nz], read only; d_p
 * device FP32 data [nx][ny][nt], overwritten.  Asynchronous on the plan's
 * stream.                                                                    */
pai_status pai_forward_plan(const pai_geometry* g, void* cuda_stream, pai_plan_t* out);
pai_status pai_forward_model(pai_plan_t plan, const float* d_f, float* d_p);
/* Box extents of a forward-model plan (by = 1 in 2-D).                       */
pai_status pai_forward_box(pai_plan_t plan, int* bx, int* by, int* bz);

/* Smooth cutoff of the data (Eq. data-part, Sec. 2; built as in Sec. 5):
 * partial (limited-view) data are g = w_cut * (Q f), the complete data times
 * a smooth nonnegative weight that is one well inside the measured region
 * and falls to zero at its edges.
 *
 * Definition.  Positions are measured in sampling steps along every data
 * axis (lateral axes in units of dx (dy), time in units of dt); the data grid
 * [nx] ([ny]) [nt] spans the box [0, n_a] on axis a, its samples sitting at
 * 0 .. n_a - 1.  The mollifier is phi(v) = C exp(-1 / (1 - |v|^2/eps)^4) for
 * |v|^2 < eps, zero elsewhere, C making its integral one (the support and
 * exponent of Sec. 5, written scale-free; eps is in squared sampling steps,
 * the support radius sqrt(eps) steps).  w_cut(u) = integral of
 * phi(v) chi_box(u - v) dv.  A sample whose distances to the lower and upper
 * faces of axis a are s_a = min(u_a, n_a - u_a) has the weight
 * T[s_1]..[s_d] with every s_a clipped to R = ceil(sqrt(eps)) (beyond that
 * distance the face does not reach the mollifier); the (R+1)^d table is
 * computed on the host by Gauss-Legendre quadrature (error below 1e-9).
 *
 * pai_cutoff_table: host only, no device work.  dim 2 or 3; 1 <= eps <= 256.
 * Writes R to *R (may be NULL) and, when table != NULL and capacity >=
 * (R+1)^dim, the weights, index ((s_x (R+1) + s_y) (R+1) + s_t) in 3-D and
 * s_x (R+1) + s_t in 2-D; a smaller capacity returns PAI_ERR_INVALID_ARG
 * after writing *R.
 *
 * pai_set_cutoff: attaches the cutoff with parameter eps to a single-problem
 * plan (reconstruction or forward model); eps = 0 removes it.  Requires
 * 1 <= eps <= 256 and every data axis n_a >= 2 ceil(sqrt(eps)) (so each
 * sample is within reach of at most one face per axis), else
 * PAI_ERR_INVALID_ARG; batched plans return PAI_ERR_UNSUPPORTED.  Computes
 * the table, uploads it into plan-owned device memory and waits for the
 * upload.  A forward-model plan with a cutoff returns w_cut * (Q f) from
 * pai_forward_model: the weight is applied by the kernel that copies the
 * detector rows out of the box, at no extra memory traffic.
 *
 * pai_cutoff: d_out = w_cut * d_in over the plan's data grid [nx][ny][nt]
 * (device FP32, contiguous).  d_in == d_out (in place) touches only the
 * samples whose weight differs from one; partially overlapping buffers are
 * not allowed.  PAI_ERR_INVALID_ARG without a cutoff set.  Asynchronous on
 * the plan's stream.                                                         */
pai_status pai_cutoff_table(int dim, double eps, double* table, int capacity, int* R);
pai_status pai_set_cutoff(pai_plan_t plan, double eps);
pai_status pai_cutoff(pai_plan_t plan, const float* d_in, float* d_out);

/* Size of the static device scratch array used by pai_spectrum_rows_noalloc. */
#define PAI_NOALLOC_SCRATCH_BYTES (1u << 20)

/* The fused row stage of pai_spectrum (prescale, oversampled FFT, window
 * gather and weight for every lateral-frequency row) for ONE problem, with no
 * device allocation at all.  The paper has no counterpart: this entry point
 * exists for callers that may not call cudaMalloc / cudaFree (processes whose
 * device memory is already reserved by another allocator or pool, real-time
 * loops in which an allocation's implicit synchronisation is not allowed).
 * g:      problem statement, as for pai_plan (host, read during the call).
 * d_pt:   device, interleaved complex64 lateral spectrum rows [rows][nt], the
 *         output of an unnormalised real-to-complex FFT of p over the lateral
 *         axes with the last lateral axis halved: rows = nx/2+1 (2-D) or
 *         nx*(ny/2+1) (3-D).  Read only.
 * d_fhat: device, interleaved complex64 [nx][ny][nz/2+1], overwritten with the
 *         same half spectrum pai_spectrum returns.
 * cuda_stream: cudaStream_t (NULL = legacy default stream).
 * Scratch: every table, descriptor and the work counter live in one static
 * device array of PAI_NOALLOC_SCRATCH_BYTES bytes that each GPU loading the
 * library holds until exit; geometries whose tables exceed it return
 * PAI_ERR_UNSUPPORTED, checked on the host before any CUDA call and before the
 * pointers are looked at.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress).  Each call fills its tables in a host
 * buffer and copies them into the array with a cudaMemcpyAsync on cuda_stream
 * (from pageable memory: the driver stages the bytes before the call returns),
 * zeroing the work counter; the copy is ordered after the stream's earlier
 * work, so consecutive calls on one stream are safe.  The array keeps the last
 * call's contents, and calls that overlap on the GPU (other streams, other
 * threads) race on it.
 * Calls no cudaMalloc, cudaFree or allocating library routine.              */
pai_status pai_spectrum_rows_noalloc(const pai_geometry* g, const float* d_pt, float* d_fhat, void* cuda_stream);

/* Static description of a status code; never NULL.                           */
const char* pai_status_string(pai_status s);

#ifdef __cplusplus
}
#endif

#endif /* PAI_H */
