/*
 * sfft.h - C ABI of the GB300 (sm_103a) difference-imaging library.
 *
 * The library fits a science CCD S against its aligned reference R with the
 * model used by the paper's image-differencing step (Sec. 2.3.2, with the
 * method as introduced in Sec. 1: a Fourier-domain formulation with a
 * delta-function kernel basis that follows spatial PSF variations):
 *
 *     S'(x) ~ sum_j K_j(x) R~(x - u_j) + B'(x),
 *     K_j(x) = sum_p theta[j N_K + p] phi_p(x),
 *     B'(x)  = sum_q theta[L^2 N_K + q] psi_q(x),
 *
 * with u_j the L x L offsets (j = (u_y + w) L + (u_x + w), w = (L-1)/2),
 * phi_p (psi_q) the monomials xt^a yt^b of total degree <= D_K (D_B) in
 * xt = 2x/(W-1) - 1, yt = 2y/(H-1) - 1, ordered by degree and, within a
 * degree, by decreasing a; N_K = (D_K+1)(D_K+2)/2, N_B likewise, and
 * N = L^2 N_K + N_B unknowns.  The fit minimises
 * sum_x M_fit(x) [S'(x) - model(x)]^2 where M_fit is 1 on pixels at least w
 * from every edge whose whole L x L footprint is good; bad pixels are
 * bad[x] != 0, non-finite R or non-finite S.  R_m = good ? R - s_R : 0 and
 * S' = S - s_S with sky constants (s_R, s_S).
 *
 * Conventions shared by every entry point:
 *  - Images are row-major [batch][H][W] (row y, column x), batch stride H*W.
 *  - All image, matrix and status pointers are DEVICE pointers unless stated.
 *    The caller owns every buffer; the library never frees them.
 *  - Every call is asynchronous on the plan's stream: it enqueues kernels and
 *    returns.  Argument and shape errors are returned synchronously; data
 *    errors (singular or non-finite system, wait time-out) are written per CCD
 *    into the device `info` array and never trap.
 *  - No call allocates device memory after sfft_plan; scratch lives in the
 *    caller-allocated workspace `ws` of sfft_workspace_bytes() bytes (256-byte
 *    aligned).  A workspace must not be shared by calls that overlap on the GPU.
 *  - Requirements: L odd, 1 <= L <= 11; 0 <= D_K, D_B <= 2; H >= L;
 *    16 <= W <= 2048.  The sky offsets are absorbed exactly by the background
 *    when D_B >= D_K or with SFFT_FLAG_CONST_RATIO; otherwise the fit is that
 *    of the sky-subtracted images (see sfft_solve for the reported units).
 *
 * Constant photometric ratio (SFFT_FLAG_CONST_RATIO; the constrained
 * delta-basis kernel of the literature cited in Sec. 1): the kernel sum
 * sum_j K_j(x) is one constant a_0 over the chip.  The fit is solved in the
 * basis K = a_0 delta_0 + sum_{u != 0} sum_p c[u,p] phi_p (delta_u - delta_0),
 * (L^2 - 1) N_K + 1 + N_B unknowns, i.e. the normal equations
 * (T A T^T) theta_c = T b with theta = T^T theta_c; A, b and theta keep the
 * full N-term layout above.
 *
 * The paper gives no equations for the fit; the exact definition above, the
 * mask and sky-offset semantics and the polynomial coordinates are this
 * library's reading of it.
 */
#ifndef SFFT_GB300_H
#define SFFT_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sfft_plan_s* sfft_plan_t;

typedef enum {
  SFFT_OK = 0,
  SFFT_ERR_ARG = 1,          /* invalid argument or shape (returned synchronously) */
  SFFT_ERR_CUDA = 2,         /* a CUDA runtime call failed */
  SFFT_ERR_NOMEM = 3,        /* plan-time host or device allocation failed */
  SFFT_ERR_SINGULAR = 4,     /* per-CCD info: normal matrix not positive definite */
  SFFT_ERR_NONFINITE = 5,    /* per-CCD info: non-finite normal matrix or solution */
  SFFT_ERR_TIMEOUT = 6,      /* per-CCD info: a bounded device wait gave up */
  SFFT_ERR_UNSUPPORTED = 7   /* shape or degree outside the supported range */
} sfft_status_t;

typedef enum {
  SFFT_PREC_FP64 = 0,        /* FFTs, products, partial sums and apply in FP64 */
  SFFT_PREC_MIXED = 1        /* FP32 FFTs/products/partials (KK products with split operands on the
                                tensor cores: hi x hi in TF32 plus two BF16 corrections, about
                                2^-18 per product); FP64 accumulation and refinement; Cholesky
                                factor and substitutions in FP32, every solution refined against
                                the FP64 system (see sfft_solve) */
} sfft_prec_t;

#define SFFT_FLAG_GRAPH 1u        /* sfft_subtract replays a captured CUDA graph */
#define SFFT_FLAG_CONST_RATIO 2u  /* kernel sum constant over the chip (constrained fit) */
#define SFFT_FLAG_FMA_CONTRACT 4u /* mixed path: KK contraction on the FP32 FMA pipes instead of the
                                     split TF32/BF16 products on the tensor cores (the default) */
#define SFFT_FLAG_MMA_SYNC_CONTRACT 8u /* mixed path: the tensor-core KK contraction with warp-level
                                          mma.sync instead of tcgen05 (the default) */
#define SFFT_FLAG_PAIR_LANE_CONTRACT 16u /* mixed path: the tcgen05 KK contraction with one tensor-memory
                                            lane per (difference, u_y) pair instead of one lane per
                                            difference with the u_y shifts taken from the weight rows
                                            (the default when a difference batch holds at least
                                            min(96, all) differences) */

typedef struct {
  int32_t H, W;              /* image rows, columns */
  int32_t L;                 /* kernel size (odd) */
  int32_t DK, DB;            /* kernel / background polynomial degrees */
  int32_t batch;             /* CCD pairs per call */
  int32_t prec;              /* sfft_prec_t */
  int32_t autotune;          /* 1: time contraction tile shapes at plan time and keep the fastest */
  int32_t d_batch;           /* kernel-offset differences per product/FFT pass (0 = auto) */
  int32_t rows_per_cta;      /* rows of one contraction partial sum (0 = auto) */
  int32_t lag_parts;         /* threads sharing the lags of one contraction k-slot: 2 or 3 (0 = auto;
                                FP32 path only, the FP64 path uses 2) */
  uint32_t flags;            /* SFFT_FLAG_* */
  int32_t ccd_group;         /* CCDs whose product spectra are held at once (0 = auto: every difference of a
                                CCD in one pass when its spectra fit 64 GB, as many CCDs as 32 GB of
                                product spectra hold) */
} sfft_desc_t;

/* Create a plan: validates the descriptor, builds offset/monomial/lag tables,
 * allocates the plan's small constant device tables (twiddles) and, with
 * autotune=1, times contraction tile shapes on synthetic data in its own
 * temporary buffers.  `cuda_stream` is a cudaStream_t (NULL = legacy default
 * stream).  On success *out owns the plan; release with sfft_plan_destroy. */
sfft_status_t sfft_plan(const sfft_desc_t* desc, void* cuda_stream, sfft_plan_t* out);
void          sfft_plan_destroy(sfft_plan_t plan);
sfft_status_t sfft_plan_set_stream(sfft_plan_t plan, void* cuda_stream);
int64_t       sfft_num_unknowns(sfft_plan_t plan);          /* N */
size_t        sfft_workspace_bytes(sfft_plan_t plan);       /* bytes for `ws` */
/* KK-contraction engine the plan runs: 0 FP64 FMA (FP64 path), 1 FP32 FMA,
 * 2 tensor cores through mma.sync, 3 tcgen05 with one tensor-memory lane per
 * (difference, u_y) pair, 4 tcgen05 with one lane per difference; -1 for a
 * null plan. */
int32_t       sfft_plan_engine(sfft_plan_t plan);
/* Chosen tile shape after planning: out[0] = d_batch, out[1] = rows_per_cta,
 * out[2] = lag parts of the contraction. */
sfft_status_t sfft_plan_tiles(sfft_plan_t plan, int32_t* out3);
/* CCDs per product-spectrum pass (the group the offset-difference product
 * spectra are formed and contracted for at once); -1 for a null plan. */
int32_t       sfft_plan_ccd_group(sfft_plan_t plan);
/* Failure detection (no counterpart in the paper).  The FP64 factorisation
 * separates its block steps by a grid-wide barrier whose wait is bounded:
 * after `tries` polls (each at least 64 ns) a CTA gives up, every CCD of the
 * call gets SFFT_ERR_TIMEOUT in `info` and the kernel returns with the
 * context intact.  The default (about a second) applies after plan creation
 * and again for tries < 0; small values let a test make the wait run out.
 * The barrier is a software flag wait with no asynchronous copies or
 * tensor-core work in flight, so giving up leaves nothing pending. */
sfft_status_t sfft_plan_set_wait_limit(sfft_plan_t plan, int32_t tries);
/* Wait attribution of the difference-lane contraction kernel (a profiling
 * aid; no counterpart in the paper).  In a library built with
 * -DSFFT_DLANE_WAIT_PROFILE, lane 0 of every warp of k_contract_dlane adds the
 * clock cycles it spent in each kind of wait to a device array: out[0] copy
 * warp waiting for a free stage of probe rows, [1] A producers waiting for
 * probe rows, [2] A producers waiting for a free A slot, [3] A producers
 * waiting for their tensor-memory stores, [4] B producers waiting for weight
 * rows, [5] B producers waiting for a free stage of weight-row blocks, [6] MMA
 * issuer waiting for weight-row blocks, [7] MMA issuer waiting for A operands,
 * [8] cycles of whole CTAs (thread 0).  Synchronizes the device; reset != 0
 * clears the array.  SFFT_ERR_UNSUPPORTED in the default build. */
sfft_status_t sfft_debug_contract_waits(uint64_t* out9, int32_t reset);
/* Measured FMA peak of this GPU for roofline reports (no counterpart in the
 * paper): FP32 (fp64 = 0) or FP64 (fp64 = 1) TFLOP/s = 2 x FMAs / time of a
 * kernel of independent FMA chains, 8 CTAs of 256 threads per SM, timed with
 * CUDA events on `cuda_stream` after one warm-up launch (synchronizes the
 * stream).  Allocates and frees a small device buffer for the results. */
sfft_status_t sfft_probe_fma_peak(int32_t fp64, double* tflops, void* cuda_stream);
/* Measured cost of one tcgen05 MMA with both operands in shared memory (no
 * counterpart in the paper; it bounds the stamp classifier's convolutions):
 * clock cycles per kind::f16 BF16 MMA of M = 128, K = 16 and N = n columns
 * (16 <= n <= 256, n % 16 == 0, else SFFT_ERR_ARG), canonical K-major layout
 * without swizzle, 2000 issued back to back by one thread per CTA, one CTA per
 * SM, averaged over the SMs after a warm-up launch.  SFFT_ERR_TIMEOUT if a
 * bounded completion wait gave up.  Synchronizes the stream; allocates and
 * frees a small device buffer. */
sfft_status_t sfft_probe_umma_cycles(int32_t n, double* cycles_per_mma, void* cuda_stream);
/* Number of device allocations the library's plans (and the plan-time
 * autotuner) currently hold.  For leak checks: with SFFT_FAIL_ALLOC=n set in
 * the environment, the n-th device allocation of every sfft_plan call fails
 * as a full device would (SFFT_ERR_NOMEM, message in sfft_last_error), and the
 * count returns to its value before the call. */
int64_t       sfft_debug_live_allocations(void);

/* Normal-matrix assembly (the method's Fourier-domain normal equations):
 *   A = sum_x M_fit Phi Phi^T,  b = sum_x M_fit Phi S'   (FP64 outputs)
 * KK block: for every kernel-offset difference d = u - u' and weight monomial
 * xt^a yt^b, the row-FFT cross-correlation of the masked product
 * R_m(z) R_m(z + d) with M_fit xt^a yt^b, sampled at the lags u; KB block and
 * b_K: the same with R_m against M_fit phi_p psi_q and M_fit phi_p S'; BB and
 * b_B: moments of M_fit.
 *   R, S : float [batch][H][W];  bad : uint8 [batch][H][W] or NULL (no mask);
 *   sky  : double [batch][2] = (s_R, s_S), or NULL to estimate each as the
 *          mean of the good pixels (any constant gives the same kernel and D
 *          away from non-finite pixels and the w-pixel border);
 *   A    : double [batch][N][N] (written fully, symmetric);  b : double [batch][N];
 *   ws   : workspace; keeps the masks, spectra and sky for sfft_solve/apply. */
sfft_status_t sfft_build_normal(sfft_plan_t plan, const float* R, const float* S,
                                const uint8_t* bad, const double* sky,
                                double* A, double* b, void* ws);

/* Solve A theta = b per CCD (with SFFT_FLAG_CONST_RATIO the projected
 * system T A T^T theta_c = T b, theta = T^T theta_c): Jacobi equilibration,
 * Cholesky, two triangular solves; then `refine_steps` steps of iterative
 * refinement whose residual r = sum_x M_fit Phi (S' - model) is formed in
 * image space from R and S.  The FP64 plan factors and substitutes in FP64.
 * The mixed plan factors the equilibrated matrix and substitutes in FP32; the
 * refinement steps refine that solution (their residual is b - A theta), and
 * with refine_steps = 0 one normal-equations step r = b - A theta in FP64
 * does.  theta : double [batch][N]; its
 * background part is returned in original (un-offset) units,
 * beta_q + s_S [q == 0] - s_R sum_j theta[j, q] for q < min(N_K, N_B), which
 * is B = B' + s_S - s_R sum_j K_j exactly unless D_B < D_K with a free kernel
 * sum (then the terms of degree above D_B are not representable and are left
 * out; sfft_apply with the same sky still reproduces the fitted D).
 * info : int32 [batch] (device) receives SFFT_OK / SFFT_ERR_SINGULAR /
 * SFFT_ERR_NONFINITE.  Must follow sfft_build_normal with the same ws, R, S
 * and bad. */
sfft_status_t sfft_solve(sfft_plan_t plan, const double* A, const double* b, double* theta,
                         int32_t refine_steps, const float* R, const float* S,
                         const uint8_t* bad, int32_t* info, void* ws);

/* Difference image D = S - K (x) R - B over every pixel, evaluated as
 * S' - sum_p phi_p sum_j theta[j,p] R~(x - u_j) - B'(x) with
 * R~ = finite(R) ? R - s_R : 0 and zero outside the image.
 * theta : double [batch][N] (background in original units, as sfft_solve
 * returns it); sky : double [batch][2] or NULL to reuse the workspace's sky
 * from sfft_build_normal; D : float [batch][H][W]. */
sfft_status_t sfft_apply(sfft_plan_t plan, const float* R, const float* S, const double* theta,
                         const double* sky, float* D, void* ws);

/* build_normal + solve (refine_steps) + apply in one call; with
 * SFFT_FLAG_GRAPH the enqueued work is captured once per distinct argument
 * set and replayed as a CUDA graph. */
sfft_status_t sfft_subtract(sfft_plan_t plan, const float* R, const float* S, const uint8_t* bad,
                            const double* sky, int32_t refine_steps, double* A, double* b,
                            double* theta, int32_t* info, float* D, void* ws);

/* Allocation-free difference image (no counterpart in the paper; a service for
 * callers that cannot allocate device memory - code running under a fixed
 * memory budget or inside a framework that owns all allocations - and so can
 * neither create a plan, which allocates its tables, nor supply a workspace).
 * Computes the same D as sfft_apply for the given shapes:
 *   R, S  : float [batch][H][W];  theta : double [batch][N] (background in
 *   original units, as sfft_solve returns it);  sky : double [batch][2]
 *   (required: there is no workspace to take it from);  D : float [batch][H][W];
 *   prec  : sfft_prec_t (FP32 or FP64 convolution);  cuda_stream : cudaStream_t.
 * Scratch: a fixed device array of 46848 doubles (375 KB) built into the
 * library, held on every GPU that loads it until the process exits; calls with
 * batch * N above that return SFFT_ERR_UNSUPPORTED.  The first call on each
 * device looks up that array's device address (cudaGetSymbolAddress) with the
 * device current; make that first call before any stream capture.  All calls
 * share the one array, so calls that overlap on the GPU (different streams or
 * threads without ordering) race and corrupt each other's results; the array
 * keeps the last call's contents, and every call overwrites what it reads
 * before reading it.  It calls no cudaMalloc or cudaFree. */
sfft_status_t sfft_apply_noalloc(int32_t H, int32_t W, int32_t L, int32_t DK, int32_t DB, int32_t batch,
                                 int32_t prec, const float* R, const float* S, const double* theta,
                                 const double* sky, float* D, void* cuda_stream);

/* Kernel coefficient maps for inspection: K[ccd][j] at pixel (x, y) of every
 * CCD, from theta (device) into K (device, double [batch][L*L]). */
sfft_status_t sfft_kernel_at(sfft_plan_t plan, const double* theta, double x, double y, double* K);

/* Per-phase device timing (not part of the method; instrumentation for
 * roofline reports).  When enabled, every later call records CUDA events on
 * the plan's stream around each phase; sfft_profile_read synchronizes the
 * stream, then returns accumulated milliseconds and kernel-launch counts per
 * phase (arrays of SFFT_PROF_N) and optionally resets them.  Phases are not
 * timed while the stream is being captured into a graph.  Launch counts are
 * kept whether or not timing is enabled. */
enum {
  SFFT_PROF_PREP = 0,        /* sky, masks, erosion, moments */
  SFFT_PROF_FFT_WEIGHTS = 1, /* row FFTs of weight maps, R_m and residual maps */
  SFFT_PROF_FFT_PROD = 2,    /* row FFTs of the products R_m(z) R_m(z + d) */
  SFFT_PROF_CONTRACT_KK = 3, /* lag contraction of the product spectra (KK block) */
  SFFT_PROF_CONTRACT_RK = 4, /* lag contraction against R_m spectra (KB, b_K, refinement) */
  SFFT_PROF_SCATTER = 5,     /* assembly of A and b from the accumulators */
  SFFT_PROF_SOLVE = 6,       /* Cholesky, triangular solves (and, mixed with no refinement steps,
                                one FP64 residual step) */
  SFFT_PROF_APPLY = 7,       /* convolve-and-subtract and refinement residual */
  SFFT_PROF_LAG_DFT = 8,     /* tensor-core KK paths: lags u_x over the k-slot products and the
                                exact slot-0 sums */
  SFFT_PROF_N = 9
};
sfft_status_t sfft_profile_enable(sfft_plan_t plan, int32_t enable);
sfft_status_t sfft_profile_read(sfft_plan_t plan, double* ms, int64_t* launches, int32_t reset);

const char* sfft_status_str(sfft_status_t s);
/* Last CUDA error text seen by the library on this thread ("" if none). */
const char* sfft_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SFFT_GB300_H */
