/*
 * gs.h -- C ABI of the GB300 generalized-sampling library (libgs.so).
 *
 * Generalized sampling (Jacobsen, Nielsen, Rasmussen, "Generalized Sampling in
 * Julia"): from Fourier samples w^s_m = f-hat(xi_m), m = 1..M, estimate the
 * coefficients of f in the boundary-corrected Daubechies scaling-function basis
 * V_J^int of [-1/2, 1/2] (Sec. 3.3, eq. modified_Daubechies_span) or of its
 * tensor square (Sec. 5) by weighted least squares (Sec. 2, eq. least_squares;
 * Sec. 4.1, eq. weighted_least_squares).  The library applies the change-of-basis
 * matrix T (Sec. 4, eq. CoB_block_1D; Sec. 5, eq. 2Dwavelet_border_division;
 * App. C) and its adjoint without forming it, and solves the least-squares
 * problem with CGLS (Sec. 6.3).
 *
 * Conventions (all entry points)
 *   - Complex values are interleaved (re, im): complex128 = 2 doubles,
 *     complex64 = 2 floats.
 *   - Coefficients: 1D vector of N = 2^J values, index i = 0..N-1 is the
 *     function phi^int_{J, i - N/2} (left edge functions first, Sec. 3.3);
 *     2D array of N*N values stored x-fastest: X(i, j) at i + N*j, i along x
 *     (App. C's column-major vec; Sec. 5).
 *   - Samples: M values in the caller's order of xi.
 *   - Rows of T carry the density weight sqrt(mu_m) (Sec. 4.1).  Data passed to
 *     gs_solve must already be weighted: y_m = sqrt(mu_m) * f-hat(xi_m).
 *   - Device pointers are CUDA device (or managed) memory owned by the caller;
 *     host pointers are read during the call only.  "stream" is a cudaStream_t
 *     (NULL = legacy default stream); all device work of a call is ordered on it.
 *   - No call synchronises the device except gs_plan_* (which return after the
 *     tables are built) and gs_solve (which reads its stop flag).
 *   - Errors are returned as gs_status; gs_last_error_detail() gives a
 *     thread-local description.  Nothing aborts or throws across the ABI.
 *   - A plan is not thread-safe: do not run two calls on one plan concurrently.
 *
 * Environment switches (diagnostics and tests; leave them unset in normal use)
 *   GS_NO_TC      2D float32 spread and interpolation run the scalar kernels
 *                 instead of the tensor-core ones (read at every launch)
 *   GS_DF64       every 2D float64 forward apply interpolates in double-float
 *                 arithmetic, not only the refinement residual's (read at every
 *                 launch)
 *   GS_NO_GRAPHS  solves launch their kernels one by one instead of through
 *                 captured CUDA graphs (read once per process)
 *   Results agree within the tolerances stated at each entry point either way.
 */
#ifndef GS_H
#define GS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gs_plan_s* gs_plan;

typedef enum {
  GS_OK = 0,
  GS_EINVAL = 1,        /* bad argument (sizes, NULL, non-finite xi or weights) */
  GS_ENOMEM = 2,        /* device or host allocation failed */
  GS_ECUDA = 3,         /* a CUDA runtime call failed (detail has the CUDA error) */
  GS_ENOTCONV = 4,      /* gs_solve hit maxit before the tolerance */
  GS_EBREAKDOWN = 5,    /* CGLS breakdown: ||T p|| = 0 or a non-finite step */
  GS_ETIMEOUT = 6,      /* a bounded device wait gave up */
  GS_EUNSUPPORTED = 7   /* a valid request the library does not implement */
} gs_status;

/* Arithmetic of one apply. */
typedef enum {
  GS_FP64 = 0, /* complex128 in and out, float64 arithmetic, KB half-width kb_m_hi */
  GS_FP32 = 1  /* complex64 in and out, float32 arithmetic, KB half-width kb_m_lo  */
} gs_precision;

/* Plan options; pass NULL for the defaults in brackets. */
typedef struct {
  int kb_m_hi;  /* Kaiser-Bessel half-width m in 2..8 (taps per dim 2m) for GS_FP64 applies [8] */
  int kb_m_lo;  /* Kaiser-Bessel half-width m in 2..8 for GS_FP32 applies [4] */
  int sigma;    /* oversampling factor of the NFFT grid, 2 or 4 [2] */
  int direct;   /* 1: evaluate T entry by entry (O(M N^d) per apply, small problems);
                   0: NFFT path; -1: choose (direct when M * N^d <= 2^16) [-1] */
  int chunk;    /* NFFT path: samples per work item of the spread and interpolation at
                   most; a tile's samples split into near-equal items (load balance).
                   > 0: that size; 0: 512; -1: autotune at plan time (times float32
                   T and T^H for sizes 128..1024 and keeps the fastest) [0] */
  int lattice;  /* NFFT path on the lattice (1/sigma) Z^d: when sigma xi is an integer for
                   every sample and dimension (e.g. the uniform grids of Sec. 3.2, tensor
                   grids in 2D), T and T^H are exact FFTs: the grid value of each sample is
                   picked (T) or folded in (T^H) with no window and no deapodisation.
                   0: use it when the samples allow; 1: never; 2: require it (GS_EINVAL
                   otherwise) [0] */
} gs_opts;

/* Build a 1D plan: the representation of T (paper: Freq2Wave(xi, "dbp", J[, bandwidth]),
 * Sec. 6.1-6.2).  Validation: p in 1..6 (p = 1 is Haar), 2^J >= 2p (Sec. 3.3),
 * J <= 20, M >= 1, xi finite.
 *   out        receives the plan (NULL on error)
 *   xi         host, M sampling frequencies (any order, any range; Sec. 3.1)
 *   p, J       vanishing moments and scale: N = 2^J coefficients
 *   bandwidth  > 0: density weights mu = 1D Voronoi cell lengths, outer cells
 *              closed by [-bandwidth, bandwidth] (Sec. 4.1); <= 0: mu = 1
 *   weights    host, M density weights mu_m >= 0 (overrides bandwidth), or NULL
 *   stream     cudaStream_t for the table-building kernels */
gs_status gs_plan_1d(gs_plan* out, const double* xi, int64_t M, int p, int J,
                     double bandwidth, const double* weights, const gs_opts* opts,
                     void* stream);

/* Build a 2D plan (Sec. 5, App. B, App. C).  xi is host, M x 2 interleaved
 * (xi_x, xi_y); weights is host M or NULL (mu = 1). */
gs_status gs_plan_2d(gs_plan* out, const double* xi, int64_t M, int p, int J,
                     const double* weights, const gs_opts* opts, void* stream);

void gs_plan_destroy(gs_plan plan);

/* Sizes of a plan: dims (1 or 2), M, N (per dimension), ncoef (N or N*N). */
gs_status gs_plan_sizes(gs_plan plan, int* dims, int64_t* M, int64_t* N, int64_t* ncoef);

/* y = T x (Sec. 4, eq. CoB_block_1D; Sec. 5; App. C: interior by NFFT, corners
 * and sides by the boundary factors).
 *   x  device, ncoef complex (complex128 for GS_FP64, complex64 for GS_FP32)
 *   y  device, M complex of the same type; overwritten */
gs_status gs_apply_T(gs_plan plan, int precision, const void* x, void* y, void* stream);

/* x = T^H y (Sec. 3.2 adjoint NDFT; App. C adjoint).  Buffers as gs_apply_T. */
gs_status gs_apply_TH(gs_plan plan, int precision, const void* y, void* x, void* stream);

/* x = T^H y like gs_apply_TH, for callers that must not allocate device memory
 * while they run (code recording a CUDA graph, runtimes with a fixed memory
 * arena).  The paper has no counterpart; it is a deployment variant.  The spread
 * scratch lives in a fixed 8 MiB device array reserved by the library on every
 * device that loads it; the call allocates nothing.  NFFT-path plans only
 * (GS_EUNSUPPORTED for direct mode); GS_EINVAL when the plan's scratch exceeds
 * 8 MiB (nwork * part_stride complex values).  All calls share the array, so
 * calls whose GPU work overlaps race: order them on one stream.  The first call
 * on a device looks up the array address (cudaGetSymbolAddress) and keeps it for
 * the life of the process; make that first call before any stream capture.  The
 * kept address, like every plan, does not survive cudaDeviceReset (or any other
 * destruction of the device's primary context).  Buffers as gs_apply_TH. */
gs_status gs_apply_TH_noalloc(gs_plan plan, int precision, const void* y, void* x, void* stream);

/* Solver settings for gs_solve. */
typedef enum {
  GS_SOLVE_FP64 = 0,  /* textbook CGLS with GS_FP64 applies throughout */
  GS_SOLVE_MIXED = 1  /* iterative refinement: x += d, d from a CG pass on the normal
                         equations T^H T d = T^H r with GS_FP32 applies and float64
                         scalars; r = y - T x with a forward apply from float64 data
                         between passes (2D NFFT plans: its interpolation in
                         double-float arithmetic, ~1e-13 relative); T^H r (the pass
                         rhs and the stop test) with a GS_FP32 adjoint when
                         tol >= 1e-7, else GS_FP64.  Data and coefficients must stay
                         within the float32 range (|values| < 1e38). */
} gs_solve_mode;

typedef struct {
  double tol;     /* stop when ||T^H (y - T x)|| <= tol * ||T^H y|| [1e-6] */
  int maxit;      /* total CGLS iteration cap [1000] */
  int mode;       /* gs_solve_mode [GS_SOLVE_MIXED] */
  int x0_given;   /* 1: x holds a starting guess on entry, kept only if ||T^H (y - T x0)|| <
                     ||T^H y|| (else the solve starts from x = 0); 0: start from x = 0 [0] */
  int max_outer;  /* refinement passes in GS_SOLVE_MIXED [8] */
  double inner_rtol; /* GS_SOLVE_MIXED: a pass stops when its ||T^H (r - T d)|| falls
                        by this factor (or below tol ||T^H y|| / 2); the first pass of a
                        kept starting guess ends at the first inner_rtol^k ||T^H y|| below
                        its start; 0 = default [1e-3] */
} gs_solve_opts;

typedef struct {
  int iterations;     /* CGLS iterations, all passes */
  int outer;          /* refinement passes (1 in GS_SOLVE_FP64) */
  double rel_normres; /* ||T^H (y - T x)|| / ||T^H y|| at exit: x and r = y - T x in FP64,
                         T^H r in the stop-test precision of the mode */
  double rel_res;     /* ||y - T x|| / ||y|| at exit */
  int status;         /* gs_status of the solve */
} gs_solve_info;

/* Weighted least squares x = argmin ||T x - y|| (Sec. 2, eq. least_squares; the
 * paper's T \ y, Sec. 6.2) by CGLS, stopped on the normal-equation residual.
 * GS_EINVAL unless the plan has more samples than coefficients (M > N^d: Sec. 2
 * takes N < M for a stable reconstruction); applies accept any M >= 1.
 *   y    device, M complex128 (weighted data)
 *   x    device, ncoef complex128; the solution (and the start if x0_given)
 *   info host, may be NULL
 * Returns GS_ENOTCONV when maxit is reached (x holds the last iterate). */
gs_status gs_solve(gs_plan plan, const void* y, void* x, const gs_solve_opts* opts,
                   gs_solve_info* info, void* stream);

/* B independent least-squares solves (one plan each, plans distinct) with the
 * options of gs_solve.  With GS_SOLVE_MIXED and tol >= 1e-7 each solve runs as one
 * CUDA graph (nested while-conditional nodes: refinement passes around CG
 * iterations, float64 residual and stop test on the device); the B graph launches
 * are assigned up front to 16 library-owned streams, ordered after `stream`, by
 * longest-processing-time-first on an estimated cost (CG iterations of the plan's
 * previous solve times a per-iteration time model), and the call waits once, when
 * all have finished.  Other options run gs_solve per problem on those streams as
 * they come free.  y[i], x[i] as in gs_solve; infos (host, B entries) may be NULL.
 * A plan's first batch call synchronises the device once and rebuilds its cached
 * graphs: in a batch, and in every later call on that plan, the 2D spread and
 * reductions launch without overlapping the kernel before them (early-launched
 * CTAs would hold SM space the other problems' kernels can use).
 * Returns the first non-OK status of any problem (GS_ENOTCONV included). */
gs_status gs_solve_batch(const gs_plan* plans, int B, const void* const* y, void* const* x,
                         const gs_solve_opts* opts, gs_solve_info* infos, void* stream);

/* 2D density weights (App. B, eq. Voronoi_tesselation): mu[m] = area of the
 * Voronoi cell of xi_m within Y_K = [-K, K]^2, and *delta (may be NULL) = the
 * largest distance from a point of Y_K to its nearest sample (the density of
 * App. B, attained at a cell vertex).  Exact cells, computed on the GPU (one thread
 * per sample clipping the square by the bisectors of nearby samples, stopped by
 * the security radius).  xi host M x 2 interleaved, every coordinate within
 * [-K, K] (GS_EINVAL otherwise); mu host M.  Repeated points share one cell each
 * in full (their bisector is empty).  Synchronises `stream`; allocates and frees
 * its own device memory.  GS_EUNSUPPORTED if a cell needs more than 64 vertices.
 * The result suits gs_plan_2d's weights. */
gs_status gs_voronoi_2d(const double* xi, int64_t M, double K, double* mu, double* delta, void* stream);

/* ---- Learned warm start (an addition beside the paper's method) ----------
 * A residual CNN x0 = u + f(u) on the 2-channel image (real, imaginary part) of
 * u = T^H y, pixel (j, i) = coefficient i + N j, images NCHW float32.  f is
 * `depth` 3x3 convolutions (zero padding) with `channels` hidden channels and
 * ReLU between them; the last layer starts at zero (untrained net = identity).
 * Training: float32 weights, Adam, mean-squared error; inference: bfloat16 or
 * float32 weights, float32 accumulation.  H, W multiples of 16; channels 8, 16
 * or 32; weights initialised He-uniform from `seed`. */
typedef struct gs_cnn_s* gs_cnn;
gs_status gs_cnn_create(gs_cnn* out, int H, int W, int channels, int depth, int max_batch, uint64_t seed,
                        void* stream);
void gs_cnn_destroy(gs_cnn net);
/* x0 = u + f(u) for B images (device, B x 2 x H x W float32 each) */
gs_status gs_cnn_forward(gs_cnn net, const float* u, float* x0, int B, int use_bf16, void* stream);
/* one Adam step on B (u, target) pairs; mean-squared error of x0 before the step into *loss */
gs_status gs_cnn_train_step(gs_cnn net, const float* u, const float* target, int B, float lr, double* loss,
                            void* stream);
/* loss and gradients (weights then biases, the gs_cnn_weights order) without an update */
gs_status gs_cnn_gradients(gs_cnn net, const float* u, const float* target, int B, float* grad_host, double* loss);
/* all weights then all biases, layer by layer ([c_out][c_in][3][3], [c_out]); *count always set */
gs_status gs_cnn_weights(gs_cnn net, float* host, int64_t* count);
gs_status gs_cnn_set_weights(gs_cnn net, const float* host, int64_t count);

/* Batched least squares from learned starts: for each problem the start of
 * gs_solve_learned (x0 = rms(u) net(u / rms(u)), u = T^H y[i]), then gs_solve_batch
 * with x0_given = 1 (each start kept only if ||T^H (y - T x0)|| < ||T^H y||, else
 * that problem starts from zero).  All plans 2D with the network's N x N grid; other
 * arguments as gs_solve_batch.  The paper has no counterpart (an addition beside the
 * method). */
gs_status gs_solve_batch_learned(const gs_plan* plans, int B, gs_cnn net, const void* const* y, void* const* x,
                                 const gs_solve_opts* opts, gs_solve_info* infos, void* stream);

/* A training pair for the network: u_img = image of u / rms(u), u = T^H y
 * (float32 adjoint), and, when x and x_img are non-NULL, x_img = image of
 * x / rms(u) (x: ncoef complex128, e.g. the method's reconstruction).  Images are
 * 2 x N x N float32 on the device. */
gs_status gs_cnn_pair(gs_plan plan, const void* y, const void* x, float* u_img, float* x_img, void* stream);

/* Least squares from the learned warm start: u = T^H y (float32), x0 = rms(u) *
 * net(u / rms(u)) (bfloat16 weights), then gs_solve from x0 -- or from zero when
 * ||T^H (y - T x0)|| >= ||T^H y||: the plain method is the fallback, and its
 * residual decides.  2D plans whose N x N grid is the network's image.  *used_warm_start
 * (may be NULL) tells which start was taken.  Other arguments as gs_solve. */
gs_status gs_solve_learned(gs_plan plan, gs_cnn net, const void* y, void* x, const gs_solve_opts* opts,
                           gs_solve_info* info, int* used_warm_start, void* stream);

/* Host-only (no CUDA call): the plan-time constants for p vanishing moments, so
 * they can be checked without a GPU.  h: 2p filter taps h_k, k = -p+1..p, with
 * sum 1 (App. A).  For p >= 2 also the edge matrices of App. A.1, row-major:
 * U_left, U_right (p x p, = H / sqrt2), V_left, V_right (p x (2p-1), = h / sqrt2,
 * columns m = p..3p-2) and v1(0) for both sides (p each).  Any of the output
 * pointers may be NULL.  GS_EINVAL for p outside 1..6. */
gs_status gs_boundary_constants(int p, double* h, double* U_left, double* V_left, double* v0_left,
                                double* U_right, double* V_right, double* v0_right);

/* Tracing.  gs_profile(1) makes every later kernel launch of the library (any
 * plan, any thread) record a CUDA event pair around itself on its stream;
 * gs_profile(0) stops recording.  gs_profile_report waits for the recorded
 * events, writes {"kernel name": [launches, total_ms], ...} as JSON into buf
 * (len bytes) and clears the record.  Off by default; recording adds two event
 * records per launch. */
gs_status gs_profile(int on);
gs_status gs_profile_report(char* buf, int64_t len);

const char* gs_strerror(gs_status s);
const char* gs_last_error_detail(void);

#ifdef __cplusplus
}
#endif
#endif /* GS_H */
