/*
 * zbc.h -- C ABI of the Tucker-compressed VSIE coupling-matrix library (GB300, sm_103a).
 *
 * The library implements the hot path of Giannakopoulos et al., "Compression of
 * volume-surface integral equation matrices via Tucker decomposition for magnetic
 * resonance applications" (arXiv 2103.06393): column assembly of the coil-body
 * coupling matrix Z (q*n_v x m), column-wise Tucker compression (Sec. III.A), ACA
 * and Algorithm 3 (Sec. III.C), and the products Y = Z X (Algorithm 1) and
 * Psi = Z^H Phi (Algorithm 2, Sec. III.B).
 *
 * Conventions shared by every call
 *  - Complex numbers are interleaved (re, im): complex64 = 2 x float, complex128 = 2 x double.
 *  - Matrices are column-major with an explicit leading dimension (ld >= rows).
 *  - Voxel index v = i1 + n1*(i2 + n2*i3) (column-major reshape of a column, Fig. 2);
 *    row index of Z is k*n_v + v for field component k = 0..q-1 (Y = [Y^1; ...; Y^q]).
 *  - Voxel centres are ((i - (n-1)/2) * h) per axis (grid centred at the origin).
 *  - Every pointer is a DEVICE pointer owned by the caller unless its name ends in
 *    _host.  The library never frees caller memory.
 *  - Every call returns an int status (ZBC_OK = 0, negative on error); on error
 *    zbc_last_error() returns a message (thread-local, valid until the next call on
 *    the same thread).  No C++ exception crosses this boundary.
 *  - Calls taking a stream enqueue their kernels on it and return without waiting,
 *    except where the comment says the call synchronises (compression sizes its
 *    output from device results and therefore waits).
 *  - A zbc_handle is library-owned, immutable after creation except where noted, and
 *    must not be used by two calls that overlap on the GPU (the product calls keep
 *    per-handle workspace).
 */
#ifndef ZBC_H
#define ZBC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; 0 is the legacy default stream. */
typedef struct CUstream_st* zbc_stream;

enum {
  ZBC_OK = 0,
  ZBC_EINVAL = -1,    /* bad argument: null pointer, size out of range, ld too small */
  ZBC_ENOMEM = -2,    /* device or host allocation failed */
  ZBC_ECUDA = -3,     /* a CUDA runtime call or kernel launch failed */
  ZBC_ETOL = -4,      /* a tolerance could not be met (fallback exhausted) */
  ZBC_ETIMEOUT = -5,  /* a bounded device wait gave up (kernel returned an error status) */
  ZBC_ENAN = -6,      /* NaN or Inf found in an input */
  ZBC_EIO = -7        /* file read/write failed or file is not a zbc handle */
};

typedef enum { ZBC_C64 = 0, ZBC_C128 = 1 } zbc_dtype;

/* Arithmetic form of the product kernels.
 * FP32_SIMT : complex FP32 on CUDA cores (the plain form).
 * TF32X3    : tensor cores, tcgen05 kind::tf32, each operand split hi+lo, 3 products, FP32 accumulation.
 * BF16X3    : tensor cores, tcgen05 kind::f16 with bf16 operands split into 3 terms
 *             (hi+mid+lo), the 6 products above 2^-24, FP32 accumulation.
 * TC2       : (forward only) the last mode product of the decompression on the tensor cores
 *             too: Z = U1 W per column as a tcgen05 MMA with fp16 hi+lo operands (W scaled by a
 *             power of two per tensor), chained through TMEM into the BF16X3 contraction.
 * TC_MODE1  : the products regrouped so that the mode-1 product is a dense tcgen05 GEMM
 *             (fp16 hi+lo operands scaled by powers of two, 3 products, FP32 accumulation).
 *             Adjoint: T = U1^H Phi^k per group of 128 (column, rank) rows, then
 *             Psi_j = sum conj(W) T over (rank, i2, i3) on CUDA cores (i1 tiles of 160
 *             beyond n1 = 224).
 *             Forward: per block of 128 (i2 i3, RHS) rows and i1 tile of at most 96,
 *             Y^k = U1 (W X) over all (column, rank) rows, W X generated on CUDA cores, the
 *             tensor-core sum folded into FP32 every 192 rows.
 * TC_DC     : (forward only) decompression then contraction per voxel block: Z for 32 i1 x 4T i23
 *             voxels and a chunk of 8 stored columns from U1 and the cached W on CUDA cores
 *             (FP32, written as fp16 hi + lo), the contraction with X as a tcgen05 GEMM
 *             (M = 128 voxels, N = 2 x 16 .. 2 x 128 right-hand sides, 3 products, FP32
 *             accumulation folded into an FP32 sum in tensor memory every 64 columns).
 * AUTO      : the form (and CTA shape) zbc_tune measured fastest for this handle and this
 *             right-hand-side class; before any tuning, BF16X3 for the forward product when
 *             p >= 8 and FP32_SIMT otherwise.  Every form meets the same 1e-5 relative accuracy,
 *             but their last bits differ, so AUTO results depend on the tuning. */
typedef enum {
  ZBC_FP32_SIMT = 0,
  ZBC_TF32X3 = 1,
  ZBC_BF16X3 = 2,
  ZBC_AUTO = 3,
  ZBC_TC2 = 4,
  ZBC_TC_MODE1 = 5,
  ZBC_TC_DC = 6
} zbc_precision;

typedef enum { ZBC_HOSVD = 0, ZBC_RANDOMIZED_LEARNED = 1, ZBC_RANDOMIZED_FIXED = 2 } zbc_tucker_method;

typedef enum { ZBC_ACA_DENSE_U = 0, ZBC_ACA_ALG3 = 1 } zbc_aca_mode;

typedef struct {
  int32_t n1, n2, n3;   /* voxels per axis */
  double h;             /* voxel edge (m) */
  double mask_radius;   /* voxels with sqrt(x^2+y^2) > mask_radius are zero rows; <= 0: no mask */
  double mask_box;      /* voxels with max(|x|, |y|) > mask_box are zero rows; <= 0: no mask.  A box
                           mask is a product of per-axis indicators, so it leaves the Tucker ranks
                           of a column's tensors as they are on the kept box */
} zbc_grid;

typedef struct {
  int32_t m;              /* number of segments (columns of Z) */
  const double* centre;   /* device, m x 3 row-major (x,y,z per segment), metres */
  const double* tangent;  /* device, m x 3 row-major, unit vectors */
  const double* length;   /* device, m, metres */
} zbc_segments;

typedef struct zbc_handle zbc_handle;

typedef struct {
  int32_t n1, n2, n3, q;
  int32_t M;          /* stored columns: m (Tucker only) or r_c (ACA + Tucker) */
  int32_t m;          /* columns of Z */
  int32_t has_v;      /* 1 if Z = U V^H with V (m x M) stored dense */
  int32_t max_rank;   /* largest Tucker rank over all tensors and modes */
  int64_t pool_bytes; /* bytes of cores + factors (complex64) */
  int64_t v_bytes;    /* bytes of V (complex64) */
} zbc_info;

typedef struct {
  int32_t n_tensors;   /* tensors compressed by this call */
  int32_t n_fallback;  /* randomized tensors that failed the check and were redone by HOSVD */
  int32_t max_rank;
  double max_rel_err;  /* largest certified relative Frobenius error bound over the tensors */
} zbc_compress_stats;

/* Last error message of this thread ("" if none). */
const char* zbc_last_error(void);

/* Library version string. */
const char* zbc_version(void);

/* Number of CUDA kernels this library has launched in this process (all entry points).
 * Lets a caller count the launches inside a timed region. */
int64_t zbc_kernel_launches(void);

/*
 * vsie_assemble_columns -- columns of the coupling matrix (Sec. III.A; Eq. n6, Eq. nNt).
 *   Z[(k,v), e] = h^3 len_e [ (I + grad grad / k0^2) g(r_v - c_e) t_e ]_k,
 *   g(R) = exp(-i k0 R) / (4 pi R),  k0 = 2 pi freq_hz / 299792458,
 * i.e. the point-matched (one point per voxel and per segment) dyadic kernel, evaluated
 * in FP64.  q must be 3 (piecewise-constant basis, three field components).
 *   cols : device int32[ncols], column indices e in [0, s->m)
 *   out  : device, (q*n_v) x ncols, column-major, leading dimension ld >= q*n_v, dtype dt
 * Masked voxels (grid mask_radius) give exact zeros.  A segment centre closer than
 * 1e-12 m to a voxel centre is a caller error that the kernel does not check (R = 0).
 * Entries of cols outside [0, s->m) produce an all-zero output column.
 */
int vsie_assemble_columns(const zbc_grid* g, const zbc_segments* s, double freq_hz,
                          const int32_t* cols, int ncols, int q,
                          void* out, int64_t ld, zbc_dtype dt, zbc_stream stream);

/* Green's function operator of the coupling matrix: N (Eq. nNt, the dyadic kernel above, the
 * electric-field coupling) or K (Eq. nKt, the curl of the single-layer potential, the
 * magnetic-field coupling Z_bc of the paper's GMT application). */
typedef enum { ZBC_OP_N = 0, ZBC_OP_K = 1 } zbc_operator;

/*
 * vsie_assemble_columns_op -- vsie_assemble_columns with a choice of operator and a
 * Gauss-Legendre rule of nq points (1 .. 16) along each segment:
 *   Z[(k,v), e] = h^3 len_e sum_q (w_q / 2) [ Kern(r_v - p_q) t_e ]_k,
 *   p_q = c_e + xi_q len_e t_e / 2   ((xi_q, w_q) the rule on [-1, 1]),
 *   N: Kern t = (I + grad grad / k0^2) g t,   K: Kern t = grad g x t = g' (Rhat x t),
 *   g' = -g (i k0 + 1/R).
 * q = 3: piecewise-constant basis (one point per voxel).  q = 12: piecewise-linear basis (Sec.
 * II.A): per voxel phi_0 = 1, phi_1..3 = (x - x_c)/h, (y - y_c)/h, (z - z_c)/h for each field
 * component, integrated over the voxel with the 2 x 2 x 2 Gauss-Legendre rule (the result is
 * h^3 x the rule's mean); row block b = 3 l + k (basis l, component k), row b n_v + v; ld >= 12 n_v.
 * nq = 1, q = 3 with ZBC_OP_N is exactly vsie_assemble_columns.  Arguments, layout and errors as
 * there; ZBC_EINVAL for an unknown operator, nq outside [1, 16] or q not 3 or 12.  A quadrature
 * point closer than 1e-12 m to a voxel's quadrature point is a caller error the kernel does not
 * check.
 */
int vsie_assemble_columns_op(const zbc_grid* g, const zbc_segments* s, double freq_hz,
                             const int32_t* cols, int ncols, int q, zbc_operator op, int nq,
                             void* out, int64_t ld, zbc_dtype dt, zbc_stream stream);

/* Rank-predictor MLP of the learned compression (declared with its calls below). */
typedef struct zbc_mlp zbc_mlp;

/*
 * Inputs of the randomized Tucker methods of tucker_compress (no counterpart in the paper; see
 * tucker_compress_randomized for the method).  Per (tensor t = j*q + k, mode g) the sketch width is
 *   ZBC_RANDOMIZED_LEARNED : ceil(exp(mlp(features[j])[3k + g])) + oversample (q must be 3;
 *                            zbc_rank_widths), the predictor's log-rank output for component k, mode g;
 *   ZBC_RANDOMIZED_FIXED   : fixed_width for every tensor and mode;
 * either way clamped to [2, min(n_g, lmax, 64)] and made even.
 */
typedef struct {
  const zbc_mlp* mlp;       /* LEARNED: the trained predictor */
  const float* features;    /* LEARNED: device float32, ncols x 7 row-major (zbc_mlp input layout) */
  int32_t oversample;       /* LEARNED: added to the predicted rank, 0 .. 64 */
  int32_t fixed_width;      /* FIXED: width of every (tensor, mode), >= 1 */
  const void* sketch1;      /* device complex64 Gaussian test matrices Omega_g, N_g x lmax column-major */
  const void* sketch2;      /*   (N_1 = n2 n3, N_2 = n1 n3, N_3 = n1 n2; unfolding order as in */
  const void* sketch3;      /*   tucker_compress_randomized) */
  int32_t lmax;             /* columns of each sketch, 2 .. 64 */
} zbc_rank_model;

/*
 * tucker_compress -- column-wise Tucker compression (Sec. III.A, Fig. 2; truncated HOSVD of
 * Sec. II.B.1 with De Lathauwer's bound).
 *   cols     : device, (q*n_v) x ncols column-major (ld >= q*n_v), dtype in_dt; q = 1 .. 12
 *              components per column (3: piecewise-constant basis; 12: the piecewise-linear basis
 *              of vsie_assemble_columns_op)
 *   tol      : per-tensor relative Frobenius tolerance; mode g keeps the smallest r_g with
 *              sum_{i>r_g} sigma_i^2 <= (tol^2/3) ||A||_F^2 (so ||A - A~||_F <= tol ||A||_F)
 *   method   : ZBC_HOSVD (FP64 two-pass Gram + Jacobi eigensolver per unfolding; model may be
 *              NULL), or ZBC_RANDOMIZED_LEARNED / ZBC_RANDOMIZED_FIXED (the randomized range finder
 *              of tucker_compress_randomized with the widths of `model`, and the HOSVD as the
 *              fallback of every tensor whose widths fail the tolerance check); the error bound
 *              tol ||A||_F holds for every method
 *   model    : the randomized methods' inputs (zbc_rank_model); required by them, ignored by HOSVD
 *   store_dt : storage type of cores and factors; only ZBC_C64 (the products compute in FP32 on
 *              complex64 tensors; the paper stores complex128).  ZBC_C128 gives ZBC_EINVAL.
 *   out      : *out == NULL -> a new handle holding these ncols columns;
 *              *out != NULL -> the columns are appended to that handle (same grid and q)
 *   stats_host : optional (may be NULL); n_fallback counts randomized tensors redone by HOSVD
 * Synchronises the stream (ranks size the storage).  ZBC_EINVAL on bad arguments.
 */
int tucker_compress(const void* cols, int64_t ld, int ncols, const zbc_grid* g, int q,
                    zbc_dtype in_dt, double tol, zbc_tucker_method method, const zbc_rank_model* model,
                    zbc_dtype store_dt, zbc_handle** out, zbc_compress_stats* stats_host, zbc_stream stream);

typedef struct {
  int32_t rank;             /* r_c: columns of U and V */
  int32_t converged;        /* 1 if the stopping test |x||y| <= tol sqrt(s) was met */
  int32_t row_restarts;     /* all-zero residual rows skipped (masked voxels) */
  int32_t max_tucker_rank;  /* largest Tucker rank of the compressed U */
  int32_t tucker_fallbacks; /* RANDOMIZED_FIXED: tensors of U redone by HOSVD */
  int32_t reserved;
  double s2;                /* running estimate of ||U V^H||_F^2 */
  double last_term;         /* |x||y| of the last appended column */
  double max_tucker_err;    /* largest HOSVD error bound (relative) over the tensors of U */
} zbc_aca_stats;

/*
 * aca_compress -- Z ~ U V^H by partially pivoted ACA (Sec. II.B.2), then U column-wise in
 * Tucker form (Sec. III.A), or directly Algorithm 3 (Sec. III.C: U assembled compressed, rows
 * of U by element-wise Tucker evaluation, residual columns by Algorithms 1 and 2).
 *   Rows and columns of Z come from the same point-matched kernel as vsie_assemble_columns.
 *   tol        : ACA stopping tolerance eps (|x||y| <= eps sqrt(s_k))
 *   max_rank   : upper bound on r_c
 *   mode       : ZBC_ACA_DENSE_U (dense U in HBM, complex128, compressed at the end) or
 *                ZBC_ACA_ALG3 (U never dense; each new column compressed at tucker_tol)
 *   tucker_tol : Tucker tolerance for U's tensors; <= 0 selects 3*tol (Algorithm 3's choice)
 *   method     : how U's tensors are compressed: ZBC_HOSVD (the paper's truncated HOSVD; model may
 *                be NULL) or ZBC_RANDOMIZED_FIXED (no counterpart in the paper: the certified
 *                randomized range finder of tucker_compress with model->fixed_width for every
 *                tensor and mode and the HOSVD as each failing tensor's fallback; the same
 *                tucker_tol bound).  ZBC_RANDOMIZED_LEARNED is refused: U's columns are residual
 *                columns, not single segments, so the rank predictor has no inputs for them.
 *   model      : zbc_rank_model (sketches, lmax, fixed_width) for ZBC_RANDOMIZED_FIXED
 *   out        : new handle with U (Tucker, r_c columns) and V (m x r_c) -- Z = U V^H
 *   pivots_host: optional int32[2*max_rank]: (row, column) pivot pairs in order
 * Pivots, norms and the stopping test are FP64.  Ties pick the lowest index; rows and columns
 * already used are excluded; the start row is 0 and an all-zero residual row (masked voxel)
 * moves to the next unused row.  Synchronises the stream every iteration.
 */
int aca_compress(const zbc_grid* g, const zbc_segments* s, double freq_hz, int q, double tol, int max_rank,
                 zbc_aca_mode mode, double tucker_tol, zbc_tucker_method method, const zbc_rank_model* model,
                 zbc_handle** out, zbc_aca_stats* stats_host, int32_t* pivots_host, zbc_stream stream);

/*
 * tucker_compress_randomized -- column-wise Tucker compression by a fixed-width randomized range
 * finder with an HOSVD fallback (no counterpart in the paper; Halko-Martinsson-Tropp range finder
 * per mode, as in the randomized HOSVD of Minster-Saibaba-Kilmer).  Per tensor t = j*q + k and
 * mode g: Y = A_(g) Omega_g[:, :w] (FP64 sketch), Q = orth(Y) (FP64 Householder),
 * C = A x1 Q1^H x2 Q2^H x3 Q3^H, e^2 = ||A||^2 - ||C||^2 (FP64).  If e^2 > tol^2 ||A||^2 the
 * tensor is recompressed by truncated HOSVD (counted in stats n_fallback); otherwise C is
 * truncated by HOSVD with the remaining budget (tol^2||A||^2 - e^2)/3 per mode and U_g = Q_g W_g,
 * so ||A - A~||_F <= tol ||A||_F either way.
 *   widths_host : int32[3*ncols*q], width w for (tensor t, mode g) at 3t+g; clamped to
 *                 [2, min(n_g, lmax, 64)] and made even (rounded up when room allows)
 *   sketch1/2/3 : device complex64 Gaussian test matrices Omega_g, (N_g x lmax) column-major with
 *                 N_1 = n2 n3 (unfolding column c = i2 + n2 i3), N_2 = n1 n3 (c = i1 + n1 i3),
 *                 N_3 = n1 n2 (c = i1 + n1 i2); shared by all tensors
 *   out         : as tucker_compress (new handle or append)
 * Synchronises the stream.
 */
int tucker_compress_randomized(const void* cols, int64_t ld, int ncols, const zbc_grid* g, int q, zbc_dtype in_dt,
                               double tol, const int32_t* widths_host, const void* sketch1, const void* sketch2,
                               const void* sketch3, int lmax, zbc_handle** out, zbc_compress_stats* stats_host,
                               zbc_stream stream);

/*
 * Tucker compression of columns from a few of their fibres (3D cross-Tucker): the alternative the
 * paper names for tensors too large to assemble whole for the HOSVD (end of Sec. II.B.1 and Sec. V,
 * after the linear-time Tucker approximation of Oseledets, Savostyanov and Tyrtyshnikov 2008).
 * Per tensor (column j, row block k), in FP64:
 *   index sets I_g per mode; I_2, I_3 start as s0 indices floor((2l+1) n_g / (2 s0)), l < s0;
 *   each sweep visits g = 1, 2, 3 with a < b the other modes:
 *     F_g = the n_g x |I_a||I_b| mode-g fibres through every pair of I_a x I_b;
 *     left singular pairs of F_g (two-pass Gram / Jacobi, as tucker_compress);
 *     r_g = the smallest r with sum_{i>r} s_i^2 <= ((tol/4)^2 / 3) ||F_g||_F^2, capped at rmax
 *           (the HOSVD rule on the sampled fibres at a quarter of the tolerance);
 *     I_g = the first w_g = min(r_g + over, n_g, |I_a||I_b|) rows chosen by greedy pivoting
 *           (Gaussian elimination taking the row of largest modulus) on the leading w_g
 *           singular vectors;
 *   after `sweeps` sweeps the factor U_g is the leading r_g singular vectors of the last F_g and
 *   the core interpolates the tensor on the cross J_g = the first r_g pivots of I_g:
 *     G = A[J_1, J_2, J_3] x1 M_1^-1 x2 M_2^-1 x3 M_3^-1,  M_g = U_g[J_g, :]  (r_g x r_g).
 * The entries evaluated grow linearly with the grid's side; the error is not certified (unlike
 * the HOSVD's bound) and is estimated on caller-chosen check fibres.
 */
typedef struct {
  int32_t sweeps;  /* alternating sweeps, 1 .. 16 (0: 2) */
  int32_t s0;      /* initial index-set size of modes 2 and 3, 1 .. 64 (0: 8) */
  int32_t over;    /* pivots kept per mode beyond the rank, 0 .. 16 (a NULL params: 4) */
  int32_t rmax;    /* largest rank per mode, 1 .. 64 (0: 64) */
} zbc_cross_params;

typedef struct {
  int64_t entries;        /* tensor entries evaluated (fibres, cross, check fibres) */
  double max_check_err;   /* largest estimated relative Frobenius error (-1: no check fibres):
                             sqrt(mean over checks of n_a n_b ||fibre error||^2) / ||G||_F */
} zbc_cross_stats;

/*
 * cross_tucker_compress -- the fibre cross on columns held in device memory (the fibres are read
 * from them; the form that tests the method against the HOSVD of the same columns).
 *   cols, ld, ncols, g, q, in_dt, tol, out : as tucker_compress (grid sizes even, <= 1024)
 *   params      : NULL for the defaults {2, 8, 4, 64}
 *   checks_host : host int32[nchecks][3], check fibre (g, i_a, i_b): the mode-g fibre through
 *                 index i_a of mode a and i_b of mode b (a < b the other modes), the same for
 *                 every tensor; nchecks in [0, 4096]
 *   stats_host  : optional; max_rel_err is max_check_err below (an estimate, not a bound)
 *   xstats_host : optional
 * Synchronises the stream.  ZBC_EINVAL on bad arguments (message via zbc_last_error).
 */
int cross_tucker_compress(const void* cols, int64_t ld, int ncols, const zbc_grid* g, int q, zbc_dtype in_dt,
                          double tol, const zbc_cross_params* params, const int32_t* checks_host, int nchecks,
                          zbc_handle** out, zbc_compress_stats* stats_host, zbc_cross_stats* xstats_host,
                          zbc_stream stream);

/*
 * cross_tucker_assemble -- the fibre cross with every entry evaluated from the Green's function
 * (Eq. nNt / Eq. nKt, the same evaluation as vsie_assemble_columns_op): no column is ever
 * assembled, so the memory is that of the fibres.
 *   g, s, freq_hz, q (3 or 12), op, nq : as vsie_assemble_columns_op (grid sizes even, <= 1024)
 *   cols_host   : host int32[ncols], segment indices in [0, s->m)
 *   tol, params, checks_host, nchecks, out, stats_host, xstats_host : as cross_tucker_compress
 * Synchronises the stream.
 */
int cross_tucker_assemble(const zbc_grid* g, const zbc_segments* s, double freq_hz, const int32_t* cols_host,
                          int ncols, int q, zbc_operator op, int nq, double tol, const zbc_cross_params* params,
                          const int32_t* checks_host, int nchecks, zbc_handle** out,
                          zbc_compress_stats* stats_host, zbc_cross_stats* xstats_host, zbc_stream stream);

/*
 * Rank-predictor MLP (no counterpart in the paper): 7 -> 64 -> 64 -> 64 -> 9 with ReLU, trained
 * on the GPU on log Tucker ranks.  Inputs per column (row-major, float32): segment centre / 0.1 m
 * (3), unit tangent (3), distance to the voxel box / 0.1 m (1).  Outputs: log(rank) of
 * component k, mode g at index 3k + g.  Weights are FP32 master copies; forward and backward use
 * the weights rounded to bf16 with FP32 arithmetic; loss = mean squared error over batch and
 * outputs; Adam (beta1 0.9, beta2 0.999, eps 1e-8) with bias correction.
 * Parameter packing (float32): W1 (64x7 row-major [out][in]), b1 (64), W2 (64x64), b2, W3 (64x64),
 * b3, W4 (9x64), b4 (9) -- zbc_mlp_num_params() values.
 */
int zbc_mlp_num_params(void);
int zbc_mlp_create(const float* params_host, int n_params, zbc_mlp** out);
int zbc_mlp_free(zbc_mlp* model);
/* master_host / bf16_host: optional float32[n_params] copies of the master and bf16-rounded weights */
int zbc_mlp_get_params(const zbc_mlp* model, float* master_host, float* bf16_host);
/* out (device, B x 9 row-major) = MLP(X (device, B x 7 row-major)) */
int zbc_mlp_forward(const zbc_mlp* model, const float* X, int B, float* out, zbc_stream stream);
/* grads (device, n_params) = d loss / d weights at the bf16 weights; loss (device scalar, optional).
 * Deterministic: per-CTA partial sums reduced in a fixed order. */
int zbc_mlp_backward(zbc_mlp* model, const float* X, const float* T, int B, float* grads, float* loss,
                     zbc_stream stream);
/* one Adam update of the master weights with gradients grads (device) */
int zbc_mlp_adam_step(zbc_mlp* model, const float* grads, float lr, zbc_stream stream);
/* steps x (backward + Adam) on the full batch; loss_hist (device, steps floats, optional) */
int zbc_mlp_train(zbc_mlp* model, const float* X, const float* T, int B, int steps, float lr, float* loss_hist,
                  zbc_stream stream);
/*
 * zbc_rank_widths -- widths for tucker_compress_randomized from the MLP: features (device,
 * ncols x 7) -> predicted log ranks -> w = ceil(exp(pred)) + oversample, clamped to [2, n_g].
 * widths_host: int32[9*ncols] in the (tensor t = 3j + k, mode g) -> 3t + g order.  Synchronises.
 */
int zbc_rank_widths(const zbc_mlp* model, const float* features, int ncols, const zbc_grid* g, int oversample,
                    int32_t* widths_host, zbc_stream stream);

/*
 * zbc_matvec -- Y = Z X (Algorithm 1, Sec. III.B).  With ACA storage (Z = U V^H) the library
 * first forms X' = V^H X (r_c x p) and runs Algorithm 1 on U (Sec. III.B, last paragraph).
 *   X : device complex64, m x p, column-major, ldx >= m
 *   Y : device complex64, (q*n_v) x p, column-major, ldy >= q*n_v; overwritten
 *   p : 1 .. 1024 right-hand sides
 */
int zbc_matvec(const zbc_handle* h, const void* X, int64_t ldx, int p, void* Y, int64_t ldy,
               zbc_precision prec, zbc_stream stream);

/*
 * zbc_rmatvec -- Psi = Z^H Phi (Algorithm 2, Sec. III.B).  With ACA storage the product on U
 * is followed by Psi = V Psi'.
 *   Phi : device complex64, (q*n_v) x p, ldphi >= q*n_v
 *   Psi : device complex64, m x p, ldpsi >= m; overwritten
 * Partial sums over voxel tiles are reduced in a fixed order (deterministic).
 * prec: ZBC_FP32_SIMT, ZBC_TC_MODE1 or ZBC_AUTO (others: ZBC_EINVAL).  TC_MODE1 keeps fp16
 * copies of Phi (16 bytes per complex entry, rounded up to whole N blocks) and partial sums in
 * per-handle workspaces.
 */
int zbc_rmatvec(const zbc_handle* h, const void* Phi, int64_t ldphi, int p, void* Psi,
                int64_t ldpsi, zbc_precision prec, zbc_stream stream);

/*
 * zbc_rmatvec_noalloc -- Psi = Z^H Phi in FP32 on CUDA cores, like zbc_rmatvec with
 * ZBC_FP32_SIMT, but without allocating any memory.  The paper has no counterpart.  It is for
 * callers that cannot allocate device memory at the moment they need the product: real-time or
 * embedded loops whose memory is fixed up front, allocator hooks that must not re-enter the
 * allocator, and code running while a stream is being captured (cudaMalloc is not permitted
 * there).  zbc_rmatvec keeps its partial sums in a per-handle buffer that grows on demand; this
 * entry point uses a fixed array instead.
 *   - Partial sums live in one scratch array compiled into the library: 16 MiB of device memory
 *     on every GPU that loads the library, held until the process exits.  Calls whose q*M*p
 *     (+ M*p for ACA storage) complex64 values exceed it are rejected with ZBC_EINVAL.
 *   - The handle's decompression cache must already exist: call zbc_matvec or zbc_rmatvec on the
 *     handle once first (that call allocates); otherwise ZBC_EINVAL.
 *   - The scratch array's device address is looked up on the first call made on each device
 *     (with that device current) and kept for the life of the process; make that first call
 *     before any stream capture begins, and do not use the library again on a device after
 *     cudaDeviceReset (the kept address would be stale).
 *   - All calls share the array and it keeps the last call's contents; each call overwrites all
 *     it reads, so it needs no clearing, but calls that overlap on the GPU race on it.
 * Arguments are those of zbc_rmatvec.
 */
int zbc_rmatvec_noalloc(const zbc_handle* h, const void* Phi, int64_t ldphi, int p, void* Psi, int64_t ldpsi,
                        zbc_stream stream);

/*
 * zbc_tune -- autotuner of the product kernels (no counterpart in the paper).  Times, on this
 * handle with p right-hand sides (zero-filled scratch operands), every variant of
 *   zbc_matvec : FP32_SIMT with 6 and with 9 compute warps per CTA, TF32X3, BF16X3, TC2, TC_MODE1, TC_DC
 *   zbc_rmatvec: FP32_SIMT with 6 and with 9 compute warps per CTA, TC_MODE1
 * and records the fastest of each for p's right-hand-side class (p = 1, 2, 3-4, 5-8, 9-16,
 * 17-32, 33-64, 65+), which ZBC_AUTO then uses (zbc_rmatvec_noalloc uses the faster SIMT shape).
 * Each variant runs once untimed, then is timed over two calls, or over one when that call took
 * more than 1.5 times the best of its direction so far (the tensor-core forms are timed first).
 * Afterwards the per-handle operands of the forms that no tuned class selects (TC_MODE1's, TC_DC's,
 * TC2's) are freed; a later call of such a form builds them again (zbc_device_bytes shows both).
 * A CUDA graph captured before this call may hold pointers to those operands: tune first, then
 * capture.
 *   times_ms_host : optional float[10], the variants' times in the order above (ms per call;
 *                   +inf for a variant that does not fit this handle)
 * Allocates scratch operands and synchronises `stream`: call it before any graph capture.
 */
int zbc_tune(zbc_handle* h, int p, zbc_stream stream, float* times_ms_host);

/*
 * zbc_product_status -- device-side status of this handle's product kernels (zbc_matvec,
 * zbc_rmatvec, zbc_rmatvec_noalloc).  The products run asynchronously on `stream`, so their
 * device-side failures are recorded in an error word of the handle:
 *   - a product kernel whose bounded wait (on its copy pipeline or on the tensor cores) gave up
 *     returns early with its output incomplete;
 *   - a NaN or Inf read from X (forward products) or Phi (adjoint products) is noted as the
 *     kernels read their inputs (the outputs then hold non-finite values; nothing stops).
 * This call synchronises `stream`, clears the word and returns ZBC_ETIMEOUT if a wait gave up,
 * else ZBC_ENAN if a non-finite input was seen, else ZBC_OK.  The paper has no counterpart.
 */
int zbc_product_status(const zbc_handle* h, zbc_stream stream);

/*
 * zbc_test_wait_limit -- test hook for the bounded waits (no counterpart in the paper).  The next
 * FP32 SIMT adjoint launch on this handle (zbc_rmatvec with ZBC_FP32_SIMT or zbc_rmatvec_noalloc)
 * allows each consumer warp `polls` polls of the wait for its first stage (40,000,000 normally);
 * polls = 0 makes that wait give up at once, so the launch takes its abort path (the copies
 * already issued are still waited for, with the normal limit) and zbc_product_status reports
 * ZBC_ETIMEOUT.  Later launches use the normal limit.
 */
int zbc_test_wait_limit(zbc_handle* h, uint32_t polls);

/* Release a handle and its device memory (NULL is accepted). */
int zbc_free(zbc_handle* h);

/* Shape and storage summary of a handle. */
int zbc_get_info(const zbc_handle* h, zbc_info* info_host);

/*
 * zbc_memory_bytes -- storage model of Table II (Sec. III.A) for this handle, in bytes at
 * complex64: tucker = sum over tensors of (r1 r2 r3 + n1 r1 + n2 r2 + n3 r3) * 8,
 * v = m * r_c * 8 (0 without ACA), full_equiv = q * n_v * m * 8.
 */
int zbc_memory_bytes(const zbc_handle* h, int64_t* tucker_host, int64_t* v_host, int64_t* full_equiv_host);

/*
 * zbc_device_bytes -- device memory this handle holds now (no counterpart in the paper; beside
 * zbc_memory_bytes' Table II model): pool = cores, factors, descriptors and V; caches = what the
 * product calls build once and keep (the decompression cache W = G x2 U2 x3 U3 with tile-blocked
 * U1, and the operands of the tensor-core forms); work = per-call workspaces grown so far
 * (partial sums, transposed right-hand sides, fp16 copies of Phi).  Any pointer may be NULL.
 */
int zbc_device_bytes(const zbc_handle* h, int64_t* pool_host, int64_t* caches_host, int64_t* work_host);

/*
 * Host import/export of the compressed storage (tests, checkpoints).
 * Tensor t = j*q + k (column j, component k) has ranks ranks_host[3t..3t+2] = (r1, r2, r3) and
 * occupies, in this order, complex64 entries:
 *   core G[a + r1*(b + r2*c)]            (r1*r2*r3)
 *   U1[i1 + n1*a], U2[i2 + n2*b], U3[i3 + n3*c]   (n_g x r_g column-major each)
 * consecutively in pool_host (tensors in order t = 0, 1, ...).  v_host is m x M column-major
 * complex64 or NULL (no ACA).  ranks must be in [1, n_g].
 */
int zbc_create_from_host(const zbc_grid* g, int q, int M, int m, const int32_t* ranks_host,
                         const void* pool_host, int64_t pool_elems, const void* v_host,
                         zbc_handle** out);
/* ranks_host: int32[3*M*q]; pool_host: complex64[pool_elems] (query sizes with zbc_get_info:
 * pool_elems = pool_bytes/8); v_host: complex64[m*M] or NULL.  Synchronises the device. */
int zbc_export_host(const zbc_handle* h, int32_t* ranks_host, void* pool_host, void* v_host);

/*
 * zbc_tc_selftest -- diagnostic of the tensor-core operand path (no counterpart in the paper):
 * D (128 x N, row-major) = A (128 x K, row-major) * B (N x K, row-major)^T computed with one
 * chain of tcgen05.mma through the shared-memory layout and descriptors of the product
 * kernels, operands rounded to fmt (0 = fp16, 1 = bf16, 2 = tf32), FP32 accumulation;
 * fmt 3 / 4 are fp16 / bf16 with A read from tensor memory (the mode-1 adjoint's form).
 * Host pointers; N in {16, 32, 48, 64}; K a multiple of 16 (fp16/bf16) or 8 (tf32), <= 64.
 * Synchronises the device.  Returns ZBC_ETIMEOUT if the MMA completion wait gave up.
 */
int zbc_tc_selftest(const float* A_host, const float* B_host, float* D_host, int N, int K, int fmt);

/* Checkpoint: flat little-endian file "ZBC1" + header + ranks + pool + V.  zbc_load creates
 * a new handle on the current device. */
int zbc_save(const zbc_handle* h, const char* path);
int zbc_load(const char* path, zbc_handle** out);

#ifdef __cplusplus
}
#endif
#endif /* ZBC_H */
