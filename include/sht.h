/*
 * sht.h -- C ABI of the GB300 spherical-harmonic transform on the nestable
 * Clenshaw-Curtis (Fejer second rule) latitude grid of Hotta & Ujiie (2018).
 *
 * Every entry point takes plain pointers and sizes.  Device pointers are
 * CUDA global-memory addresses on the device the plan was created on;
 * streams are cudaStream_t passed as void* (NULL = legacy default stream).
 * All transforms are asynchronous on the given stream; they return after
 * launching.  Errors are returned as negative sht_status codes and the
 * message of the most recent error on the calling thread is available from
 * sht_last_error().  No entry point falls back to the host: without a
 * usable CUDA device plan creation fails with SHT_ERR_CUDA.
 *
 * Data layouts (shared by every transform):
 *   grid      row-major [nfields][J][I], longitude fastest; latitude j = 0
 *             is the northernmost node theta_1 = pi/(J+1)  (Eq. cc-points);
 *             longitude i is lambda_i = 2 pi i / I            (Sec. 2).
 *   spectrum  [ncoef][nfields] interleaved complex (re, im), fields fastest;
 *             coefficient (m, n), 0 <= m <= n <= N, is row
 *             m (N+1) - m (m-1)/2 + (n - m)   (triangular truncation N,
 *             Eq. iSHT).  Only m >= 0 is stored: the fields are real, so
 *             X_n^{-m} = conj(X_n^m).  Im(X_n^0) is ignored on input and
 *             written as exactly 0 on output.
 *   precision SHT_FP64: grid double, spectrum complex double.
 *             split plans (SHT_BF16X*, SHT_FP16X*): grid float, spectrum
 *             complex float; the Legendre contractions run on the tensor
 *             cores as 2- or 3-term BF16/FP16 splits with FP32 accumulation.
 *
 * Normalisation (Eq. pnm-ortho, Eq. dFT): int_{-1}^{1} P~_n^m P~_{n'}^m dmu
 * = delta_{nn'}, no Condon-Shortley phase; the forward zonal DFT carries
 * 1/I and the inverse none, so sht_inverse(sht_forward(x)) = x for fields
 * band-limited to N when J >= 2N+1 and I > 2N (Eq. cc-condition,
 * Eq. fourier-condition).
 */
#ifndef SHT_H
#define SHT_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sht_plan_s* sht_plan_t;

typedef enum {
    SHT_FP64 = 0,   /* FP64 FFT and FP64 Legendre contraction            */
    SHT_BF16X2 = 1, /* FP32 FFT; Legendre as 2-term BF16 split products  */
    SHT_BF16X3 = 2, /* FP32 FFT; Legendre as 3-term BF16 split products  */
    SHT_FP16X2 = 3, /* FP32 FFT; Legendre as 2-term FP16 split products  */
    SHT_FP16X3 = 4  /* FP32 FFT; Legendre as 3-term FP16 split products  */
} sht_precision;
/* FP16 splits scale each row of the P~ table (at plan time) and each real
 * column of the FP32 operand (per call, from its largest magnitude) by a
 * power of two into [-1, 1), so that the narrow FP16 exponent range holds
 * the operands; x = x_1 + 2^-11 (x_2 [+ x_3]).  FP16x2 keeps ~22 bits of
 * each operand with 3 products, FP16x3 ~33 bits with 5 products; both
 * drop x_2 y_2 (weight 2^-22).  Errors are relative to the row and column
 * maxima rather than to each element. */

typedef enum {
    SHT_OK = 0,
    SHT_WARN_INEXACT = 1,    /* plan created, but J < 2N+1: the meridional
                                quadrature is not exact (Eq. cc-condition) */
    SHT_ERR_ARG = -1,        /* invalid argument (see each entry point)      */
    SHT_ERR_ALLOC = -2,      /* device or host allocation failed             */
    SHT_ERR_CUDA = -3,       /* a CUDA call or kernel launch failed          */
    SHT_ERR_NOT_NESTED = -4, /* grids do not nest (Sec. 3.2)                 */
    SHT_ERR_TIMEOUT = -5,    /* reserved: a bounded device wait gave up      */
    SHT_ERR_HANDLE = -6,     /* NULL, destroyed or foreign plan handle       */
    SHT_ERR_UNSUPPORTED = -7 /* valid request the library does not implement */
} sht_status;

/* Create a plan for truncation N on the J x I Clenshaw-Curtis grid with
 * nfields fields per call, on the current CUDA device.
 *   N >= 0; J odd and >= 1 (the parity fold of Appendix B needs the Equator
 *   node); I even and I > 2N (Eq. fourier-condition); I/2 must factor into
 *   2, 3 and 5 with I <= 8192; nfields >= 1; precision a sht_precision.
 * Builds on the device, once: the nodes (Eq. cc-points), the weights
 * (Eq. cc-wgt), the table of P~_n^m at the northern nodes by the three-term
 * recurrence (Sec. 4.1; FP64 with an extended exponent instead of the
 * paper's quadruple precision), the FFT twiddles, the split-precision
 * tables and a workspace of (N+1) * 2 * (J+1)/2 * nfields complex values.
 * The plan owns all of it.  Returns SHT_OK, SHT_WARN_INEXACT (plan valid),
 * SHT_ERR_ARG, SHT_ERR_ALLOC or SHT_ERR_CUDA; *out is set only on success. */
int sht_plan_create(int N, int J, int I, int nfields, int precision,
                    sht_plan_t* out);

/* Latitude grids. */
typedef enum {
    SHT_GRID_CC = 0,     /* Clenshaw-Curtis (Fejer's second rule), Eq. (cc-points),
                            weights Eq. (cc-wgt); nests K in 2K+1 (Sec. 3.2) */
    SHT_GRID_FEJER1 = 1  /* shifted equispaced grid of Fejer's first rule
                            (Sec. 3.3), theta_j = (j - 1/2) pi / J, Eq. (fejer1-points);
                            weights w_j = (2/J)(1 - 2 sum_{p=1}^{floor(J/2)}
                            cos(2 p theta_j)/(4p^2 - 1)): the interpolatory rule,
                            exact to degree J-1 (J for odd J).  Eq. (fejer1-wgt)
                            as printed lacks the factor 2 and is not exact. */
} sht_grid;

/* sht_plan_create on a chosen latitude grid (a sht_grid); everything else
 * as sht_plan_create.  On SHT_GRID_FEJER1 the plan has the same layouts,
 * precisions and entry points, with the same exactness condition
 * J >= 2N+1, except sht_restrict_nested: that grid does not nest
 * (Sec. 3.3), so it returns SHT_ERR_NOT_NESTED.  J must be odd, so that the
 * node j = (J+1)/2 lies on the Equator. */
int sht_plan_create_grid(int N, int J, int I, int nfields, int precision, int grid,
                         sht_plan_t* out);

/* Free a plan and its device memory (synchronises the plan's device).
 * NULL is a no-op returning SHT_OK; a destroyed handle gives SHT_ERR_HANDLE
 * as long as its memory has not been reused. */
int sht_plan_destroy(sht_plan_t plan);

/* Plan parameters; any output pointer may be NULL.  exact = (J >= 2N+1). */
int sht_plan_query(sht_plan_t plan, int* N, int* J, int* I, int* nfields,
                   int* precision, int* exact, size_t* ncoef);

/* Analysis, Eq. (dSHT) with the discretised Eq. (dFT) and Eq. (cc-quad):
 * real FFT of every latitude row (x 1/I, m <= N kept), equatorial fold
 * into symmetric/antisymmetric parts (Appendix B), then per m and parity
 * the contraction with P~_n^m(mu_j) w_j over the (J+1)/2 northern nodes.
 * grid: device, [nfields][J][I]; spec: device, [ncoef][nfields] complex.
 * Buffers must not overlap.  One plan serves one stream at a time (the
 * workspace is shared by its calls). */
int sht_forward(sht_plan_t plan, const void* grid, void* spec, void* stream);

/* Synthesis, Eq. (iSHT) via Eq. (iLT): per m and parity the contraction
 * with P~_n^m(mu_j), unfold to both hemispheres (Appendix B), then the
 * Hermitian inverse real FFT of every row (no scaling, m > N zero).
 * spec: device [ncoef][nfields] complex; grid: device [nfields][J][I]. */
int sht_inverse(sht_plan_t plan, const void* spec, void* grid, void* stream);

/* Adjoints (transposes) for the plain inner products: the sum over grid
 * points of x*y and the sum over stored coefficients of Re(conj(a) b).
 *   which = 0: adjoint of sht_forward (spectrum -> grid):
 *     x_ij = (w_j/I) sum_{m>=0} sum_n P~_n^m(mu_j) Re(a_n^m e^{i m lambda_i})
 *   which = 1: adjoint of sht_inverse (grid -> spectrum):
 *     a_n^m = c_m sum_j P~_n^m(mu_j) sum_i x_ij e^{-i m lambda_i},
 *     c_0 = 1, c_m = 2 for m >= 1, Im(a_n^0) = 0.
 * The paper defines no adjoint; these follow from Eq. (dSHT)/(iSHT).
 * in/out: device buffers with the layouts above. */
int sht_adjoint(sht_plan_t plan, int which, const void* in, void* out,
                void* stream);

/* Quadratic and cubic terms of the aliasing experiment (Sec. 4.2, steps 2
 * and 3): synthesise U, V and W from their spectra (Eq. iSHT), form
 * X_q = U V and X_c = U V W at every grid point, and analyse both
 * (Eq. dSHT, Eq. dFT, Eq. cc-quad) into spec_q and spec_c.  The products are
 * formed inside W's inverse FFT as it stores each point, so the grids are
 * read and written once more than by a plain synthesis.
 *   spec_u, spec_v, spec_w: device [ncoef][nfields] (read);
 *   grid_q, grid_c: device [nfields][J][I], caller-owned work grids that
 *     hold X_q and X_c on return;
 *   spec_q, spec_c: device [ncoef][nfields] (written).
 * Layouts and precision as sht_forward.  Five transforms on `stream`, one
 * after another on the plan's workspace.  SHT_ERR_ARG for NULL or
 * coinciding grids/spectra, SHT_ERR_UNSUPPORTED on reduced grids. */
int sht_alias_products(sht_plan_t plan, const void* spec_u, const void* spec_v,
                       const void* spec_w, void* grid_q, void* grid_c, void* spec_q,
                       void* spec_c, void* stream);

/* Restriction of a fine grid to the coarse plan's spectrum (Sec. 3.2 and
 * Appendix C): the coarse analysis of the sub-grid made of every 2^k-th
 * latitude starting from j = 2^k (1-based) and every 2^k-th longitude,
 * read in place by strided loads (no copy).  fine_grid: device
 * [nfields][J_f][I_f] with J_f = 2^k (J+1) - 1 and I_f = 2^k I of the
 * coarse plan; 1 <= k <= 8.  Returns SHT_ERR_ARG for a bad k and
 * SHT_ERR_NOT_NESTED for a plan on the shifted grid (SHT_GRID_FEJER1). */
int sht_restrict_nested(sht_plan_t coarse, const void* fine_grid, int k,
                        void* coarse_spec, void* stream);

/* Multigrid prolongation in spectral space (Appendix C): the lower-
 * resolution spectral space is a subset of this plan's, so a spectrum
 * truncated at Nc (0 <= Nc <= N; device [ncoef(Nc)][nfields] in the
 * spectrum layout and precision of the plan) is zero-padded to N and
 * synthesised on this plan's grid (device [nfields][J][I]), as
 * sht_inverse.  The first call allocates a spectrum-sized buffer that the
 * plan keeps (SHT_ERR_ALLOC if it cannot). */
int sht_prolong_spectral(sht_plan_t fine, const void* coarse_spec, int Nc, void* fine_grid,
                         void* stream);

/* The same prolongation added onto fine_grid (fine_grid += synthesis of the
 * zero-padded spectrum): the correction step of the two-grid V-cycle of
 * Appendix C, fused into the inverse FFT's store.  Arguments and errors as
 * sht_prolong_spectral; fine_grid is read and written. */
int sht_prolong_spectral_add(sht_plan_t fine, const void* coarse_spec, int Nc,
                             void* fine_grid, void* stream);

/* Multigrid restriction in grid space by injection (Appendix C): the coarse
 * plan's grid is every 2^k-th latitude (j_f = 2^k (j+1) - 1, 0-based) and
 * every 2^k-th longitude of the fine grid [nfields][2^k (J+1) - 1][2^k I]
 * (Sec. 3.2 nesting).  Plain strided copy; coarse_grid is [nfields][J][I].
 * SHT_ERR_NOT_NESTED on the shifted grid, SHT_ERR_ARG for k outside 1..8. */
int sht_inject_nested(sht_plan_t coarse, const void* fine_grid, int k, void* coarse_grid,
                      void* stream);

/* Allocation-free FP64 analysis, for callers that cannot allocate device
 * memory (no counterpart in the paper, which has no notion of memory
 * management): for example a plug-in inside an application that owns all
 * of the GPU's memory through its own pool, or code that runs where the
 * application forbids allocations.  Such a caller cannot create a plan, so
 * this call needs none: it computes the same result as sht_forward on an
 * FP64 plan of these sizes, rebuilding the nodes, weights, P~ table, FFT
 * tables and Fourier workspace in one fixed scratch array of
 * SHT_NOALLOC_SCRATCH_BYTES.  It calls no allocator.
 *   grid: device double [nfields][J][I]; spec: device complex double
 *   [ncoef][nfields]; size rules as for sht_plan_create (SHT_ERR_ARG for
 *   invalid sizes, SHT_ERR_UNSUPPORTED for an I too long for the
 *   shared-memory FFT).  Sizes whose tables and workspace exceed the
 *   scratch array are rejected with SHT_ERR_ARG and a message giving the
 *   bytes needed (T127 with J = 257, I = 512 fits up to 46 fields).
 * The scratch array lives in the library's device module, which the CUDA
 * runtime loads into a context on first use (lazily, by default): the first
 * call on a device (per context) commits the 32 MiB, which then stays until
 * the process exits.  Make that first call at start-up, before other code
 * takes the device memory; if the array cannot be loaded the call returns
 * SHT_ERR_CUDA with a message saying so.  A call that is not being captured
 * looks the array's address up in the current context; a call under stream
 * capture uses the address its context remembered from an earlier call, so
 * make the first call before any capture (SHT_ERR_ARG otherwise).
 * Every call overwrites the array: calls that overlap on the GPU race, so
 * serialise them (one stream, or events).  Each call rewrites every entry
 * it reads, so results never depend on an earlier call. */
#define SHT_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
int sht_forward_noalloc(int N, int J, int I, int nfields, const double* grid,
                        double* spec, void* stream);

/* Groups: several plans (for example uneven truncations of an ensemble, or
 * the levels of a multigrid ladder) transformed by one launch per kernel
 * stage, so that a batch is four launches per transform pair and fits in
 * one CUDA graph.  The paper has no counterpart; the per-plan results are
 * those of sht_forward / sht_inverse on each plan.
 *   plans: 1..8 live plans of one precision on one device, each at most
 *   once (their workspaces are used).  The group refers to the plans; they
 *   must outlive it.  Returns SHT_ERR_ARG or SHT_ERR_HANDLE otherwise. */
typedef struct sht_group_s* sht_group_t;
int sht_group_create(const sht_plan_t* plans, int nplans, sht_group_t* out);
int sht_group_destroy(sht_group_t group);

/* Analysis of every plan's grid: grids[q] and specs[q] are the device
 * buffers of plan q (host arrays of nplans pointers), layouts as for
 * sht_forward.  Calls of a group, and of its plans, must not overlap. */
int sht_group_forward(sht_group_t group, const void* const* grids, void* const* specs,
                      void* stream);

/* Synthesis of every plan's spectrum, as sht_inverse per plan. */
int sht_group_inverse(sht_group_t group, const void* const* specs, void* const* grids,
                      void* stream);

/* Synchronise the plan's device and report device-side failures of the
 * plan's kernels since the last call: SHT_ERR_TIMEOUT if a kernel gave
 * up on one of its bounded waits (a tensor-core pipeline stage or an
 * asynchronous copy; that call's outputs are then invalid), SHT_OK
 * otherwise.  Clears the recorded status. */
int sht_plan_status(sht_plan_t plan);

/* Launch shapes (no counterpart in the paper; they change speed, never a
 * result).  fields_per_cta: fields whose latitude rows one FFT CTA
 * transforms (1..min(nfields, 64), within 227 KB of shared memory).
 * tile_width: column-tile width of the split tensor-core GEMMs, 64 or 128
 * (split plans only; SHT_ERR_UNSUPPORTED for FP64).  A value of 0 leaves
 * that shape unchanged.  Changing the tile width synchronises the device
 * and reallocates the plan's tile lists; groups created before then
 * reject the plan (SHT_ERR_ARG) until they are recreated.  Not to be
 * called while the plan has work in flight on another stream. */
int sht_plan_set_tuning(sht_plan_t plan, int fields_per_cta, int tile_width);

/* Current launch shapes; tile_width is 0 for FP64 plans.  Either pointer
 * may be NULL. */
int sht_plan_get_tuning(sht_plan_t plan, int* fields_per_cta, int* tile_width);

/* Autotuner: time `reps` (1..1000) inverse + forward pairs per candidate on
 * `stream`, using the plan's workspace and temporary device buffers of one
 * grid and one spectrum (zero fields), first over the fields-per-CTA
 * values 1, 2, 3, 4, 5, 6, 8, 10, 12, 16 that fit, then over the tile
 * widths 128 and 64 (split plans), and keep the fastest.  The choice is
 * remembered for the process per (device, N, J, I, nfields, precision):
 * a later call for the same shape applies it without timing.  Outputs
 * (host, may be NULL): the chosen shapes and the mean milliseconds of a
 * pair under them.  Synchronous; SHT_ERR_ALLOC if the buffers cannot be
 * allocated.  The plan must not be in use on another stream meanwhile. */
int sht_plan_autotune(sht_plan_t plan, int reps, void* stream, int* fields_per_cta,
                      int* tile_width, float* ms_per_pair);

/* Reduced transform (Sec. 4.1, the option of the paper's own runs): the
 * Legendre sums neglect P~_n^m(mu_j) below 1e-16 in magnitude.  Here that is
 * done per tile and conservatively: for each (m, parity) the nodes nearer
 * the pole than the first node where some |P~_n^m| of that parity reaches
 * 1e-16 are dropped in whole 16-node K tiles of the forward contraction and
 * whole 128-node row tiles of the inverse one (those rows are written as
 * zero).  FP64 plans drop whole 16-node K chunks of the forward sums and
 * whole 32-node row tiles of the inverse ones the same way.  on = 0
 * restores the full sums.  Synchronises the device and rebuilds the plan's problem
 * and tile lists; groups that hold the plan keep working and follow the
 * setting, since the set of tiles does not change. */
int sht_plan_set_reduced(sht_plan_t plan, int on);

/* Reduced Clenshaw-Curtis grids (Sec. 6 proposes reduced and octahedral
 * grids on the Clenshaw-Curtis latitudes).  Latitude j (0-based from the
 * north) carries its own number I_lat[j] of equispaced longitudes
 * lambda_i = 2 pi i / I_lat[j].
 *
 * sht_reduced_grid_sizes applies the reduction rule Sec. 6 quotes (at
 * least 4 M_j + 1 longitudes, M_j the zonal wavenumber beyond which every
 * |P~_n^m(mu_j)| is below 1e-16) to any plan's P~ table: M_j = the largest
 * m with some |P~_n^m(mu_j)| >= 1e-16, and I_lat[j] = the smallest count
 * >= 4 M_j + 1 allowed by `rule`, capped at the plan's I.  SHT_REDUCED_SMOOTH
 * allows every even count whose half has no prime factor above 5 (fewest
 * points); SHT_REDUCED_FAST allows the counts 2 L whose half-length L has a
 * compile-time FFT kernel (128, 256, 512, 640, 1024, 1280, 2048, 2560):
 * a few more points, far faster FFTs.  I_lat: host array of J ints,
 * written.  SHT_ERR_ARG for an unknown rule.  Synchronous.
 *
 * sht_plan_create_reduced creates a plan on the Clenshaw-Curtis latitudes
 * of J nodes with I_lat[j] longitudes on latitude j (host array of J ints,
 * copied; each even and <= 8192, symmetric about the Equator; the largest
 * must exceed 2N).  Rows whose half-length has a prime factor above 5 are
 * transformed by Bluestein's chirp-z method (two FFTs of a 2-3-5-smooth
 * length >= I_lat[j] - 1), so every even count works, at a higher cost.  Grids of the
 * plan are device arrays [nfields][P] of P = sum_j I_lat[j] points, row j
 * (all its longitudes) after row j-1.  Row j carries the zonal wavenumbers
 * m <= min(N, I_lat[j]/2 - 1): the forward transform takes X^m(phi_j) from
 * the zonal DFT of the row's points (Eq. dFT with 1/I_lat[j]) and zero
 * above that range, then the quadrature of Eq. (cc-quad); the inverse
 * synthesises that range of Eq. (iSHT) on each row.  sht_forward,
 * sht_inverse, sht_adjoint (the transposes for the plain inner products),
 * sht_prolong_spectral, sht_plan_set_reduced, the tuning calls and
 * sht_plan_status take such plans; sht_restrict_nested and
 * sht_inject_nested return SHT_ERR_NOT_NESTED and grouped launches
 * SHT_ERR_UNSUPPORTED.  Errors as sht_plan_create_grid; SHT_ERR_ARG for a
 * bad I_lat.
 *
 * sht_plan_grid_points writes the points per field of any plan's grid
 * (sum_j I_lat[j] for a reduced plan, J I otherwise). */
typedef enum { SHT_REDUCED_SMOOTH = 0, SHT_REDUCED_FAST = 1 } sht_reduced_rule;
int sht_reduced_grid_sizes(sht_plan_t plan, int rule, int* I_lat);
int sht_plan_create_reduced(int N, int J, const int* I_lat, int nfields, int precision,
                            sht_plan_t* out);
int sht_plan_grid_points(sht_plan_t plan, long long* npts);

/* sht_plan_create_reduced with a zonal shift per latitude: half_shift[j] =
 * 1 puts latitude j's longitudes half a spacing east of the meridian,
 * lambda_i = 2 pi (i + 1/2) / I_lat[j], as on the tropical rows of the
 * icositetrahedral grid (Sec. 6 names the phase shift this needs in the
 * zonal transforms); 0 keeps lambda_i = 2 pi i / I_lat[j].  half_shift:
 * host array of J ints, each 0 or 1, symmetric about the Equator.  The
 * forward transform multiplies row j's X^m by e^{-i m pi / I_lat[j]}, the
 * inverse by its conjugate.  Errors as sht_plan_create_reduced. */
int sht_plan_create_reduced_shifted(int N, int J, const int* I_lat, const int* half_shift,
                                    int nfields, int precision, sht_plan_t* out);

/* Octahedral Clenshaw-Curtis grid (Sec. 6 proposes it; the counts are
 * ECMWF's octahedral pattern): the j-th latitude from either pole (j = 1 ..
 * (J+1)/2) carries first + step (j - 1) longitudes, mirrored about the
 * Equator (first = 20, step = 4 is the usual octahedral grid).  Writes
 * I_lat (host, J ints).  SHT_ERR_ARG for J even or < 1, first odd or < 2,
 * step odd or < 0, or an Equator row above 8192.  Host only. */
int sht_octahedral_grid_sizes(int J, int first, int step, int* I_lat);

/* Icositetrahedral Clenshaw-Curtis grid (Sec. 6): 24 equal-area triangular
 * panels, 6 around each pole down to 30 degrees of latitude and 12 in the
 * tropical belt.  The j-th latitude from either pole carries 6 j
 * longitudes (6 panels of j points) up to the latitude j30 = round((J+1)/3)
 * nearest 30 degrees (theta = pi/3), and 6 j30 on every tropical row; the
 * tropical rows after j30 alternate half_shift = 1, 0, 1, ... (a triangular
 * lattice).  Writes I_lat and half_shift (host, J ints each) for
 * sht_plan_create_reduced_shifted.  SHT_ERR_ARG for J even or < 1 or NULL
 * arrays.  Host only. */
int sht_icositetrahedral_grid_sizes(int J, int* I_lat, int* half_shift);

/* Copy plan tables to host memory (test and inspection aid).  Any pointer
 * may be NULL.  w: J doubles (Eq. cc-wgt, all nodes); mu: J doubles
 * (cos theta_j); pnm: ncoef x (J+1)/2 doubles, rows in spectrum order,
 * columns the northern nodes j = 0..(J-1)/2.  Synchronous. */
int sht_plan_copy_tables(sht_plan_t plan, double* w, double* mu, double* pnm);

/* Per-kernel timing (instrumentation, no counterpart in the paper).  With
 * on != 0 every kernel the plan launches is bracketed by a pair of CUDA
 * events recorded on the launch stream; off stops recording. */
int sht_profile_enable(sht_plan_t plan, int on);

/* Synchronise the recorded events and return, per stage, the summed device
 * time in milliseconds and the number of times the stage ran since the
 * last read, then reset.  ms and launches are host arrays of
 * SHT_PROFILE_STAGES entries: 0 forward FFT (+fold), 1 forward Legendre,
 * 2 inverse Legendre, 3 inverse FFT (+unfold), 4 split-precision operand
 * conversion.  sht_profile_read_kernels also writes, per stage, the number
 * of kernels the library launched inside it (kernels: host array of
 * SHT_PROFILE_STAGES entries, or NULL): a stage can be several kernels,
 * e.g. the spectrum split and the GEMM of the split inverse Legendre
 * contraction, or one launch per row length on a reduced grid. */
#define SHT_PROFILE_STAGES 8
int sht_profile_read(sht_plan_t plan, double* ms, long long* launches);
int sht_profile_read_kernels(sht_plan_t plan, double* ms, long long* launches,
                             long long* kernels);

/* Pipe throughput probe (instrumentation, no counterpart in the paper):
 * the rate of one resident wave of CTAs per SM running chains of
 * independent fused multiply-adds in registers, the ceiling against which
 * the FP64 Legendre contraction (kind 0: DFMA) and the FP32 FFT arithmetic
 * (kind 1: FFMA; kind 2: paired fma.rn.f32x2) are reported.  Calibrates its
 * trip count to about 20 ms per launch, runs `reps` (1..100) launches on
 * `stream` and writes the best rate in TFLOP/s (2 flops per FMA) to
 * *tflops (host).  Synchronous; allocates nothing; SHT_ERR_ARG for a bad
 * kind, reps or a NULL tflops, SHT_ERR_CUDA if a launch fails. */
int sht_measure_fma_peak(int kind, int reps, void* stream, double* tflops);

/* Message of the last error on this thread ("" if none). */
const char* sht_last_error(void);

/* Library version string. */
const char* sht_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SHT_H */
