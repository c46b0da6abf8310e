/*
 * bs.h -- C ABI of libbs, the GB300 (sm_103a) implementation of the
 * visibility-based multi-frequency angular bispectrum (MABS) and 3D
 * bispectrum estimator of arXiv:2506.10526, Section 3.2.
 *
 * Pipeline (each stage runs in the library's own CUDA kernels):
 *   bs_grid_load  ring (shell) masking with weights W = 1/N_g  (Eq. vg, Eq. iFT)
 *                 + inverse 2D FFT of every (ring, channel) to a real
 *                   image-plane field F (Eq. iFT; Eq. iFT_I for unit masks)
 *   bs_counts     exact integer closed-triangle counts T(i,j,l), which equal
 *                 the I-field triple sums of Eq. (estimator_t) divided by the
 *                 pixel count, and the sampling N_nu of Fig. Nv
 *   bs_mabs       triple contraction  S = sum_x F_i F_j F_l  over the image
 *                 pixels for every ring triple i <= j <= l and every ordered
 *                 channel triple of a channel block, normalised to Eq.
 *                 (estimator_t): B_A = S / (A M^2 T); optionally accumulated
 *                 into the (dnu1, dnu2) collapse of Section 3.2
 *   bs_mabs_delta folded, collapsed MABS B_A(l1,l2,l3, dnu1, dnu2)
 *   bs_bs3d       Eq. (dft): 2D DFT over (dnu1, dnu2) to (k_par1, k_par2)
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Grids are centred: element [v + nt/2][u + nt/2] holds grid point
 *    U_g = (u, v), u, v integers in [-nt/2, nt/2).  Ring m holds the cells with
 *    e_m <= |U_g| < e_{m+1} (|U_g|^2, an exact integer, compared with e^2 in
 *    FP64); U_g = 0 and cells with a component equal to -nt/2 are never binned.
 *  - Visibilities must be Hermitian, V(-U) = conj V(U) (the sky is real).  The
 *    library reads only the u >= 0 half-plane and mirrors it; bs_check_hermitian
 *    tests the assumption.
 *  - Ring triples are enumerated lexicographically over i <= j <= l:
 *    trip = 0 for (0,0,0), 1 for (0,0,1), ...  Channel triples are ordered
 *    (nu1, nu2, nu3), nu1 slowest.
 *  - "dev" pointers are CUDA device pointers on the plan's device, "host"
 *    pointers are host memory.  The caller owns every buffer passed in; the
 *    plan owns its workspace.  Device work is asynchronous on the given
 *    cudaStream_t (passed as void*; NULL = legacy default stream) unless a
 *    function says it synchronises.
 *  - Undefined estimates (no closed triangle, a flagged channel, or no sampled
 *    channel triple) are NaN.
 *  - Every function returns a bs_status.  A failure stores a message that
 *    bs_last_error returns; CUDA errors are sticky for the plan (later calls
 *    return BS_ERR_STATE) until it is destroyed.  No call falls back to a CPU
 *    path: without a usable sm_103a device, bs_plan_create returns
 *    BS_ERR_NO_DEVICE.
 *  - Not thread-safe per plan: one host thread at a time may use a plan.
 */
#ifndef BS_H_
#define BS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BS_ABI_VERSION 13

typedef struct bs_plan_s *bs_plan;

typedef enum {
    BS_OK = 0,
    BS_ERR_ARG = 1,           /* invalid argument (size, range, NULL, alignment) */
    BS_ERR_NO_DEVICE = 2,     /* no CUDA device, or not compute capability 10.3 */
    BS_ERR_CUDA = 3,          /* a CUDA runtime call or kernel launch failed */
    BS_ERR_OOM = 4,           /* device allocation failed */
    BS_ERR_NOT_HERMITIAN = 5, /* bs_check_hermitian found V(-U) != conj V(U) */
    BS_ERR_TIMEOUT = 6,       /* a bounded device-side wait gave up */
    BS_ERR_STATE = 7,         /* call out of order (e.g. no grid loaded) or sticky error */
    BS_ERR_UNSUPPORTED = 8    /* valid request this library does not implement */
} bs_status;

/* Arithmetic of the triple contraction (bs_mabs). */
enum {
    BS_PREC_FP32 = 0,       /* FP32 SIMT FMA, FP32 partial sums, FP64 across tiles */
    BS_PREC_SPLIT_BF16 = 1, /* tcgen05 tensor cores: pair and field operands split
                               into BF16 hi + lo, three products (hi.hi + hi.lo +
                               lo.hi) accumulated in FP32 TMEM, FP64 across tiles */
    BS_PREC_SPLIT_FP16 = 2  /* tcgen05 tensor cores, same three products as
                               split BF16 on FP16 hi + lo parts: each field is
                               scaled by a power of two 2^k (k per image side, ring
                               and realisation, from the field's largest |value|, so
                               that |scaled field| < 2^7) and the pair product of two
                               scaled fields stays below 2^14; the FP64 sums undo the
                               scales exactly.  Per term the rounding error is about
                               3 x 2^-22 of its magnitude (split BF16: 3 x 2^-16) at
                               the same tensor-core cost; field magnitudes within
                               2^-93 .. 2^107 keep the full precision */
};

typedef struct {
    int nt;                  /* N_t: uv grid side, even, 8..1024 */
    int nchan;               /* N_c: channels, 1..4096 */
    int nbins;               /* n_b: annular rings, 1..32 */
    const double *bin_edges; /* host, nbins+1 strictly ascending ring edges in grid
                                units of |U|; copied at create */
    int fft_m;               /* image-plane FFT side M; 0 = smallest M = 2^a 3^b 5^c,
                                M % 4 == 0, with M > 3 * (largest |u| or |v| of a
                                binned cell), which makes the pixel sum count only
                                exactly closed triangles (no wrap-around) */
    int precision;           /* BS_PREC_* */
    int batch;               /* realisations processed together, >= 1 */
    double norm_A;           /* A of Eq. (estimator_t); <= 0 means 1 */
    double r, rprime, dnu_c; /* comoving distance r, r' = dr/dnu, channel width:
                                Eq. (dft) multiplies by (r^2 r' dnu_c)^2; <= 0 means 1 */
    int multires;            /* 1: every ring triple (i,j,l) uses its own image side, the
                                smallest M = 2^a x {8, 12} with M > c_i + c_j + c_l and
                                M > 2 max(c) (c = largest |u| or |v| in a ring): closure
                                stays exact, the pixel sums shrink with the rings;
                                fields are kept at each side that some triple needs
                                (every precision; the FP32 path launches once per
                                side).  0: one M for all (fft_m rule). */
    int general;             /* 0: Hermitian visibilities and sampling (the sky is real):
                                real fields and real estimates.  1: general input -- the
                                visibilities V and the sampling N_g need not satisfy
                                V(-U) = V(U)*, N_g(-U) = N_g(U) (Eqs. iFT, iFT_I with
                                complex fields): the weighted grid X = W V is split
                                into Hermitian parts X = X_H + i Y, the real path runs on
                                X_H + t Y for t = 0, 1, -1, 2 (four internal
                                realisations per realisation), and the cubic in t gives
                                the complex S = sum_x F_i F_j F_l exactly:
                                Re S = 2 S(0) - (S(1) + S(-1)) / 2,
                                Im S = (9 S(1) - S(-1) - 2 S(2) - 6 S(0)) / 6.
                                Outputs are complex128 (interleaved re, im) with the
                                layouts of the Hermitian case; counts use the occupied
                                cells as given.  The error bound, the monopole and
                                cylindrical binnings and Monte Carlo ensembles take
                                general = 0 only (BS_ERR_UNSUPPORTED). */
    int chan_sampling;       /* 0: one sampling grid N_g for every channel (ngrid_dev
                                [nt][nt]).  1: per-channel sampling N_g(nu) (Eq. vg with
                                per-baseline flags; ngrid_dev [nchan][nt][nt] required,
                                symmetric in U for each channel): the denominator of
                                Eq. (estimator_t), sum_theta I1 I2 I3, depends on the
                                channel triple and is computed like the numerator from
                                the occupancy masks [N_g(nu) > 0] (two internal
                                realisations per realisation), to the precision of the
                                contraction; estimates are S_D / (A S_I) per channel
                                triple, and the collapse takes the ratio of the summed
                                numerators and denominators over the triples at +-d.
                                Exact integer counts (bs_counts) are geometric then.
                                Not with general = 1; the error bound and Monte Carlo
                                ensembles take chan_sampling = 0. */
} bs_plan_desc;

/* ---- checked build ---------------------------------------------------------
 * A library built with -DBS_CHECKED (libbs_checked.so) checks the indices of
 * the kernels' main global accesses against the extents of their buffers; a
 * violation is counted, the first one recorded, and the access skipped
 * instead of faulting.  bs_checked_build: 1 in such a library, else 0.
 * bs_checked_status: out_host[4] = {violations since the last reset, site of
 * the first, its index, the extent it was checked against}; reset != 0
 * clears the counters.  Synchronises.  bs_checked_selftest: one guarded
 * increment of element idx of an internal n-element buffer (1 <= n <= 4096),
 * so that a test can see an out-of-range index reported (site 0x7fff).  Both
 * return BS_ERR_UNSUPPORTED in an ordinary build. */
int bs_checked_build(void);
bs_status bs_checked_status(int reset, uint64_t *out_host);
bs_status bs_checked_selftest(int64_t n, int64_t idx, void *cuda_stream);

/* ABI version this library was built with (BS_ABI_VERSION). */
int bs_abi_version(void);

/* Create a plan on the current CUDA device.  Host-side work: ring labels,
 * alias-free FFT size, twiddle tables, ring-triple list.  Device workspace is
 * allocated lazily at the first device call, or taken from
 * bs_plan_set_workspace.  Errors: BS_ERR_ARG (desc out of range, edges not
 * ascending), BS_ERR_NO_DEVICE (no device / not sm_103), BS_ERR_UNSUPPORTED. */
bs_status bs_plan_create(const bs_plan_desc *desc, bs_plan *out);

/* Release the plan and any workspace it allocated itself.  NULL is a no-op. */
bs_status bs_plan_destroy(bs_plan plan);

/* Message of the last failure on this plan (or of the last failed
 * bs_plan_create on this thread when plan is NULL).  Never NULL. */
const char *bs_last_error(bs_plan plan);

/* Plan facts, written to info_host[0..n) (int64):
 *  [0] M (FFT side)          [1] number of ring triples T_r
 *  [2] fields per realisation (nbins*nchan)   [3] workspace bytes needed
 *  [4] u columns kept per field (largest |u| of a binned cell + 1)
 *  [5] number of ring triples with at least one closed triangle
 *      (valid after the first bs_grid_load or bs_counts), else -1
 *  [6] number of image sides (levels) the plan keeps fields at */
bs_status bs_plan_info(bs_plan plan, int64_t *info_host, int n);

/* Image side M used for each ring triple, int64 [T_r] (0: the triple's annuli
 * cannot form a triangle).  Equal to info[0] for every triple unless multires. */
bs_status bs_plan_trip_sides(bs_plan plan, int64_t *side_host);

/* Hand the plan a caller-owned device workspace of at least info[3] bytes,
 * 256-byte aligned, valid until bs_plan_destroy (e.g. a torch uint8 tensor).
 * Must be called before the first device call; otherwise the plan allocates
 * its own with cudaMalloc.  Errors: BS_ERR_ARG (too small / misaligned),
 * BS_ERR_STATE (workspace already in place). */
bs_status bs_plan_set_workspace(bs_plan plan, void *workspace_dev, size_t bytes);

/* Eq. (vg) weights + Eq. (iFT) fields for every realisation.
 *  vis_dev        complex64 [batch][nchan][nt][nt] (interleaved re, im floats),
 *                 centred, Hermitian; 8-byte aligned.
 *  ngrid_dev      float [nt][nt]: visibilities per grid cell N_g (same in every
 *                 channel); W = 1/N_g where N_g > 0, else the cell is empty
 *                 (W = 0 and it takes no part in the counts).  NULL = every
 *                 cell holds one visibility.  Plans with chan_sampling = 1:
 *                 float [nchan][nt][nt], N_g(nu) per channel (required).
 *  chan_flag_host uint8 [nchan], nonzero = channel flagged (W = 0 for the whole
 *                 channel: its triples are undefined).  NULL = none flagged.
 * Image-plane fields of side M are kept in the plan workspace.  Triangle
 * counts are recomputed when ngrid_dev is not NULL.  Resets the collapse
 * accumulators (as bs_delta_reset). */
bs_status bs_grid_load(bs_plan plan, const void *vis_dev, const float *ngrid_dev,
                       const uint8_t *chan_flag_host, void *cuda_stream);

/* Host copies of the integer counts of the last load (synchronises):
 *  tri_host  int64 [T_r]: ordered closed triangles per ring triple (or NULL)
 *  nnu_host  int64 [(2nchan-1)^2]: folded N_nu(dnu1, dnu2) of the channel
 *            triples accumulated since the last reset, indexed
 *            [(dnu1 + nchan-1)*(2nchan-1) + dnu2 + nchan-1] (or NULL). */
bs_status bs_counts(bs_plan plan, int64_t *tri_host, int64_t *nnu_host);

/* Triple contraction for one channel block (Eq. estimator_t).
 *  block_host  int32 [6] = {nu1_lo, nu1_hi, nu2_lo, nu2_hi, nu3_lo, nu3_hi},
 *              half-open channel ranges; NULL = every channel for all three.
 *  out_full_dev  double [batch][T_r][nchan][nchan][nchan] or NULL: entries of the
 *              block are overwritten with B_A (NaN where undefined); entries
 *              outside the block are left untouched.  General plans: complex128
 *              (double pairs) of the same shape.
 *  accumulate  1: add the block's pixel sums and sampling to the collapse
 *              accumulators used by bs_mabs_delta / bs_bs3d.
 *              2: the same for a cube block S x S x S (nu1, nu2 and nu3 ranges
 *              equal), using the symmetry of a ring triple with a repeated
 *              ring under exchanging that ring's channels: for (i, i, l) only
 *              nu1 <= nu2 and for (i, j, j) only nu2 <= nu3 is contracted, and
 *              the other ordering is filled in from it before the sums are
 *              read (the cube is closed under the exchange, so the result is
 *              the sum over the whole cube).  Split-precision plans without
 *              general input or per-channel sampling; out_full_dev must be
 *              NULL.  Ordinary blocks (1) may follow symmetric cubes; a
 *              symmetric cube after ordinary blocks needs bs_delta_reset.
 *              0: nothing is accumulated.
 * Errors: BS_ERR_STATE (no grid loaded; accumulate = 2 after ordinary blocks),
 * BS_ERR_ARG (block out of range, accumulate not 0..2, accumulate = 2 with a
 * block that is not a cube or with out_full_dev), BS_ERR_UNSUPPORTED
 * (accumulate = 2 on an FP32, general or per-channel sampling plan). */
bs_status bs_mabs(bs_plan plan, const int32_t *block_host, double *out_full_dev,
                  int accumulate, void *cuda_stream);

/* Zero the collapse accumulators and the accumulated sampling. */
bs_status bs_delta_reset(bs_plan plan, void *cuda_stream);

/* Raw collapse accumulators, for merging the work of several plans or ranks
 * (Section 3.2: the collapse to (dnu1, dnu2) averages over channel triples, so
 * the sums over disjoint channel blocks add, and the mean is formed once, from
 * the merged sums and sampling).
 *  sums_dev  double [batch][T_r][2nchan-1][2nchan-1]: sum over the accumulated
 *            channel triples of S = sum_x F_i F_j F_l at (nu1-nu3, nu2-nu3)
 *            (unfolded, not normalised), index [d1+nchan-1][d2+nchan-1]
 *  nnu_host  int64 [(2nchan-1)^2]: the unfolded count of accumulated valid
 *            channel triples at each separation, same index
 * bs_delta_export copies them out (either pointer may be NULL).  In a general
 * plan the batch dimension holds the four Hermitian components of each
 * realisation (4 x batch entries, component fastest), in a per-channel
 * sampling plan the numerator and occupancy components (2 x batch).
 * bs_delta_import replaces (add = 0) or adds to (add = 1) the plan's
 * accumulators; bs_mabs_delta and bs_bs3d then normalise the merged sums.
 * Plans merged this way must share the shape (grid, channels, rings, image
 * sides, precision, batch, flags and sampling), so that a ring triple's
 * normalisation A M^2 T is the same in each.
 * Errors: BS_ERR_ARG, BS_ERR_STATE (no grid loaded), BS_ERR_TIMEOUT (as
 * bs_mabs_delta, on export), BS_ERR_CUDA. */
bs_status bs_delta_export(bs_plan plan, double *sums_dev, int64_t *nnu_host, void *cuda_stream);
bs_status bs_delta_import(bs_plan plan, const double *sums_dev, const int64_t *nnu_host, int add,
                          void *cuda_stream);

/* Folded collapsed MABS (Section 3.2; fold of Fig. Nv) from the accumulated
 * blocks: for every ring triple and separation (d1, d2) in [-(nchan-1),
 * nchan-1]^2, the mean of B_A over the accumulated valid channel triples with
 * (nu1-nu3, nu2-nu3) = (d1, d2) or (-d1, -d2).
 *  out_dev  double [batch][T_r][2nchan-1][2nchan-1], index [d1+nchan-1][d2+nchan-1];
 *           the plane is point symmetric; NaN where no triple was sampled.
 *           General plans: complex128 of the same shape.
 * If a tensor-core contraction ran since the last check, synchronises on
 * cuda_stream to read its error word and returns BS_ERR_TIMEOUT when one of
 * its bounded waits gave up (the accumulated sums are then invalid). */
bs_status bs_mabs_delta(bs_plan plan, double *out_dev, void *cuda_stream);

/* Eq. (dft) applied to the folded collapsed MABS:
 *   B(a, b) = (r^2 r' dnu_c)^2 sum_{n,m} exp(-2 pi i (n a + m b)/nchan) B_A(n, m)
 * with n, m over the integers of [-nchan/2, nchan/2) -- one period of the
 * nchan-periodic kernel (the printed limits, -nchan/2 ... nchan/2, would count
 * the end separation of an even nchan twice) -- unsampled separations
 * contributing nothing, and a, b in [-nchan/2, nchan/2).  The input plane is
 * point symmetric, so the imaginary part of the sum comes only from the
 * unpaired edge n, m = -nchan/2; the real part is returned.
 * k_par a = 2 pi a / (r' nchan dnu_c).
 *  out_dev  double [batch][T_r][nchan][nchan], index [a + nchan/2][b + nchan/2].
 *           General plans: complex128 of the same shape (each of the real and
 *           imaginary parts of the folded plane transformed as above).
 * Checks the contraction's error word like bs_mabs_delta. */
bs_status bs_bs3d(bs_plan plan, double *out_dev, void *cuda_stream);

/* The same two results for the closable ring triples only (T > 0), in
 * ascending ring-triple index: n_c = bs_plan_info()[5] planes per realisation
 * instead of T_r.  The other planes of bs_mabs_delta / bs_bs3d carry no
 * information (NaN / 0), so these layouts write (and a caller copies) only
 * the planes with data.
 *  bs_mabs_delta_closable  out_dev double [batch][n_c][2nchan-1][2nchan-1]
 *  bs_bs3d_closable        out_dev double [batch][n_c][nchan][nchan]
 * Values are bit-identical to the matching planes of the full layouts
 * (complex128 for general plans).
 * Errors: as bs_mabs_delta / bs_bs3d. */
bs_status bs_mabs_delta_closable(bs_plan plan, double *out_dev, void *cuda_stream);
bs_status bs_bs3d_closable(bs_plan plan, double *out_dev, void *cuda_stream);

/* Upper bound on the rounding error of the estimates of Eq. (estimator_t)
 * computed from the last bs_grid_load, for the plan's precision.  For every
 * ring triple, beta bounds |B_A(computed) - B_A(exact)| of each of its
 * estimates: every entry of the full cube that bs_mabs writes, and (the
 * collapse being a mean) every entry of the folded plane of bs_mabs_delta.
 * The bound is worst-case and first-order: with S = sum_x F_i F_j F_l,
 *   |dS| <= (c_term + c_acc) ||F_i||_3 ||F_j||_3 ||F_l||_3
 *           + eps_fft sum over the three fields of
 *             ||F_a||_2 min(||F_b||_inf ||F_c||_2, ||F_b||_2 ||F_c||_inf)
 *   (Hoelder and Cauchy-Schwarz on the pixel sum, the normwise error of the
 *   FP32 transforms), beta = 1.01 |dS| / (A M^2 T), norms the largest over
 *   the channels of each ring's fields; u = 2^-24:
 *   c_term  FP32 u; split BF16 3 x 2^-16 + u; split FP16 3 x 2^-22 + u (plus
 *           the FP16 subnormal floor 2^-25 (2^14 + 2^7) M^2 2^-(k_i+k_j+k_l))
 *   c_acc   FP32 (1024 + ceil(M^2/1024) + 1) u; split modes
 *           2 u (3 ceil(M^2/16) + 1) (FP32 accumulation of the K16 MMAs)
 *   eps_fft (16 (ceil(log2 M) + 2) + 2) u
 * General plans (complex estimates from the real evaluations S(t) at t = 0,
 * 1, -1, 2): beta bounds the modulus of the complex error, the hypot of
 * 2 b_0 + (b_1 + b_-1)/2 (real part) and (9 b_1 + b_-1 + 2 b_2 + 6 b_0)/6
 * (imaginary part), b_t the bound above for the evaluation at t.
 * Per-channel sampling plans (R = S_D / (A S_I), collapsed as a ratio of
 * sums): the bound is per bin of the folded plane, which must be given,
 *   |R - R_exact| <= (b_D / A + |R| b_I) / (<S_I> - b_I)
 * with b_D, b_I the bound above (unnormalised) for the numerator and the
 * occupancy-field denominator and <S_I> the bin's mean computed
 * denominator (infinite where <S_I> <= b_I); bound_dev then holds, per ring
 * triple, the largest bin bound of that plane (it covers the folded plane,
 * not the full cube, whose entries each have their own denominator).
 *  bound_dev   double [batch][T_r], written; NaN for ring triples without a
 *              closed triangle
 *  delta_dev   NULL, or a folded plane as bs_mabs_delta (closable = 0:
 *              [batch][T_r][2nchan-1][2nchan-1]) or bs_mabs_delta_closable
 *              (closable = 1: [batch][n_c][2nchan-1][2nchan-1]) wrote it
 *              (double2 entries for a general plan)
 *  relerr_dev  NULL (with delta_dev NULL), or double with the entry count of
 *              delta_dev: per bin, the relative error bound beta / |B_A|
 *              (modulus for a general plan; NaN where the estimate is
 *              undefined)
 * Reads the plan's fields, so call it before the next bs_grid_load.
 * Errors: BS_ERR_ARG (NULL bound_dev, only one of delta_dev / relerr_dev,
 * no delta_dev for a per-channel sampling plan), BS_ERR_STATE (no grid
 * loaded), BS_ERR_OOM (scratch of a per-channel sampling plan), BS_ERR_CUDA. */
bs_status bs_mabs_error_bound(bs_plan plan, double *bound_dev, const double *delta_dev,
                              int closable, double *relerr_dev, void *cuda_stream);

/* Eq. (vg): nearest-grid-point gridding of raw visibilities onto the plan's
 * N_t x N_t grid, with channel pre-averaging (Section 4).  Visibility
 * (baseline i, input channel c) goes to the cell g = (floor(u_i + 1/2),
 * floor(v_i + 1/2)) (FP64) and, the sky being real, its conjugate to -g;
 * cells with |u| or |v| >= N_t/2 are dropped; input channel c feeds output
 * channel c / avg; flagged data (F = 0) are skipped.
 *  uv_dev       double [nbl][2]: baseline (u, v) in grid units
 *  vis_dev      complex64 [nbl][nchan_in]
 *  flag_dev     uint8 [nbl][nchan_in], 1 = flagged, or NULL
 *  nchan_in     avg * nchan of the plan
 *  mode 0       out_vis = V_g (sum), out_ng = N_g (count), as Eq. (vg)
 *  mode 1       out_vis = V_g / N_g, out_ng = 1 where N_g > 0 (else both 0):
 *               the input of bs_grid_load that applies the per-channel
 *               weight 1 / N_g(nu) of Eq. (vg)
 *  out_vis_dev  complex64 [nchan][N_t][N_t], centred, row index v (the
 *               layout bs_grid_load reads), overwritten
 *  out_ng_dev   float [nchan][N_t][N_t], overwritten
 * FP32 atomic sums (their order varies between runs).
 * Errors: BS_ERR_ARG (NULL, nchan_in != avg * nchan, mode). */
bs_status bs_grid_visibilities(bs_plan plan, const double *uv_dev, const void *vis_dev,
                               const uint8_t *flag_dev, int64_t nbl, int nchan_in, int avg,
                               int mode, void *out_vis_dev, float *out_ng_dev, void *cuda_stream);

/* Mean |U| of each ring's binned grid cells, in grid units (the mid point of
 * the ring's edges when it holds no cell): U_m in k_perp = 2 pi U_m / r.
 *  umean_host  double [nbins], written. */
bs_status bs_plan_ring_umean(bs_plan plan, double *umean_host);

/* Monopole of the 3D bispectrum binned in triangle size and shape (Section
 * 2, Eq. shape and Eq. bs_lm with l = m = 0; the (k1, mu, t) binning of
 * Section 5).  Samples: every closable ring triple (i, j, l) x every delay
 * pair (a, b); sides k_n = sqrt(kperp_n^2 + kpar_n^2) with kpar(a) for ring
 * i, kpar(b) for ring j and -kpar(a) - kpar(b) for ring l; k1 >= k2 >= k3,
 * t = k2 / k1, mu = -k1.k2 / (k1 k2) = (k1^2 + k2^2 - k3^2) / (2 k1 k2).
 *  b3d_dev        double [batch][n_c][nchan][nchan] as bs_bs3d_closable writes
 *                 it, or NULL: bin the model of Eq. (bsana),
 *                 2 f_ng [P(k1)P(k2) + P(k2)P(k3) + P(k3)P(k1)] with
 *                 P(k) = p_amp k^p_index, at the same discrete modes (the
 *                 binned analytic prediction [B]_d of Section 5)
 *  kperp_host     double [nbins]: k_perp of each ring (e.g. 2 pi U_m / r)
 *  kpar_host      double [nchan]: k_par of Eq. (dft) row a + nchan/2
 *                 (2 pi a / (r' nchan dnu_c))
 *  k1_edges_host  double [n_k1 + 1], finite and ascending (n_k1 <= 1024);
 *                 bin q holds e_q <= k1 < e_{q+1}
 *  n_mu, n_t      linear bins of mu and t over [0.5, 1] (<= 1024 each); the
 *                 value 1 falls in the last bin
 *  sum_dev        double [batch (1 for the model)][n_k1][n_mu][n_t]: sum of
 *                 the values in each bin (overwritten)
 *  count_dev      int64 [n_k1][n_mu][n_t]: samples in each bin (overwritten);
 *                 the monopole is sum / count
 * Side lengths from ring centres close only approximately: samples whose mu
 * or t falls outside [0.5 - 1e-2, 1 + 1e-2] are dropped, the rest clamped to
 * [0.5, 1].  The bin is decided in FP32 on squared lengths (k1 >= e_q as
 * S1 >= e_q^2, t >= tau as S2 >= tau^2 S1, mu >= m as
 * (S1 + S2 - S3)^2 >= 4 m^2 S1 S2): it equals the FP64 decision except for
 * samples whose k1 lies within a relative 1e-6 of a k1 edge, or whose t lies
 * within 1e-6 or mu within 4e-6 of a shape edge or an acceptance limit.
 * Values, sums and the model (from FP64 squared lengths) are FP64.
 * kperp_host must lie in [1e-8, 1e8] and |kpar_host| <= 1e8 (FP32 range of
 * the squared comparisons).
 * General plans: b3d_dev holds complex (double2) values and sum_dev complex
 * sums in the same layout; the binning is linear, so the real and imaginary
 * parts are binned separately (through plan scratch of about the size of
 * b3d_dev, allocated on first use and kept).  Both pointers must then be
 * 16-byte aligned.  The model (b3d_dev NULL) stays real.
 * Errors: BS_ERR_ARG (NULL, counts out of range, edges not ascending, k out
 * of range, misaligned complex pointers),
 * BS_ERR_STATE (no counts yet), BS_ERR_UNSUPPORTED (bins x realisations
 * beyond one CTA's shared memory), BS_ERR_OOM (scratch of a general plan). */
bs_status bs_bs_monopole(bs_plan plan, const double *b3d_dev, const double *kperp_host,
                         const double *kpar_host, const double *k1_edges_host, int n_k1,
                         int n_mu, int n_t, double f_ng, double p_amp, double p_index,
                         double *sum_dev, int64_t *count_dev, void *cuda_stream);

/* Multipole moments with m = 0 of the 3D bispectrum, binned like
 * bs_bs_monopole (Section 2, Eq. bs_lm with the line-of-sight direction p of
 * Eq. orient): in the triangle frame p_z = mu_1 = k_par(side 1) / k1, the
 * largest side's line-of-sight cosine, and the discrete form of Eq. (bs_lm)
 * (4 pi times the mean over a bin's samples) is
 *   B_l^0(k1, mu, t) = sqrt(4 pi (2l+1)) < Y_l^0 B > = (2l+1) < P_l(mu_1) B >.
 * m != 0 needs the azimuth of p about k1, which the triangle's handedness in
 * the sky plane fixes; side lengths from ring centres do not (and it is
 * undefined for collinear triangles).  Samples: as bs_bs_monopole but without
 * the delay row and column a, b = -nc/2 of an even nchan (their point
 * reflections lie off the grid), so that every sample's reflection
 * (a, b) -> (-a, -b) is present: mu_1 changes sign and the bin does not, and
 * the odd multipoles of a point-symmetric 3D bispectrum vanish identically.
 * mu_1 and P_l (Bonnet's recursion) are FP64; the bin is the monopole's.
 *  lmax       0..4
 *  sum_dev    double [batch][lmax + 1][n_k1][n_mu][n_t]: sums of
 *             (2l+1) P_l(mu_1) B over each bin's samples (overwritten)
 *  count_dev  int64 [n_k1][n_mu][n_t]: samples per bin (overwritten);
 *             B_l^0 = sum / count
 * Other arguments as bs_bs_monopole (b3d_dev required; complex values and
 * sums for a general plan).
 * Errors: as bs_bs_monopole; BS_ERR_ARG for lmax out of range. */
bs_status bs_bs_multipoles(bs_plan plan, const double *b3d_dev, const double *kperp_host,
                           const double *kpar_host, const double *k1_edges_host, int n_k1,
                           int n_mu, int n_t, int lmax, double *sum_dev, int64_t *count_dev,
                           void *cuda_stream);

/* The 3D bispectrum of every closable ring triple binned on an n x n grid in
 * the (k_par1, k_par2) plane (Section 5: the binning behind Fig. cylbs).
 *  b3d_dev     double [batch][n_c][nchan][nchan] as bs_bs3d_closable writes it
 *  kpar_host   double [nchan], strictly increasing: k_par of Eq. (dft) row
 *              a + nchan/2
 *  edges_host  double [n + 1] ascending, n <= 64; delay index a falls in bin
 *              q when e_q <= kpar[a] < e_{q+1} (decided on the host in FP64)
 *  sum_dev     double [batch][n_c][n][n]: sum over the (a, b) in bins (q, r)
 *  count_dev   int64 [n][n]: number of those (a, b), the same for every plane
 * Both outputs are overwritten; the binned value is sum / count.
 * General plans: complex (double2, 16-byte aligned) b3d_dev and sum_dev, as
 * for bs_bs_monopole.
 * Errors: BS_ERR_ARG, BS_ERR_STATE (no counts yet), BS_ERR_OOM (scratch of a
 * general plan). */
bs_status bs_bs_cylindrical(bs_plan plan, const double *b3d_dev, const double *kpar_host,
                            const double *edges_host, int n, double *sum_dev,
                            int64_t *count_dev, void *cuda_stream);

/* Check V(-U) = conj V(U) on every binned cell of every channel and
 * realisation: |V(-U) - conj V(U)| <= tol * max|V| (synchronises).
 * Returns BS_OK or BS_ERR_NOT_HERMITIAN. */
bs_status bs_check_hermitian(bs_plan plan, const void *vis_dev, double tol, void *cuda_stream);

/* ---------------------------------------------------------------------------
 * Batched Monte Carlo (Section 4: ensemble mean and 1-sigma of the MABS and
 * the 3D bispectrum over many realisations).  An ensemble holds shape groups
 * (uneven grid sides, channel counts and ring sets); group g processes
 * desc[g].batch realisations per run.  A run loads every group's fields,
 * contracts the full channel cube of every realisation of every group in ONE
 * persistent tensor-core launch (split BF16 or split FP16), forms the folded collapsed
 * plane and Eq. (dft), and adds each realisation to per-bin Welford
 * statistics (FP64 mean and M2).  The first run executes eagerly; later runs
 * with use_graph replay a captured CUDA graph of the same launches.
 * ------------------------------------------------------------------------- */
typedef struct bs_mc_s *bs_mc;

/* Create the ensemble: one plan per group (every desc must use the same
 * tensor-core precision, BS_PREC_SPLIT_BF16 or BS_PREC_SPLIT_FP16), device
 * input buffers, statistics.  Allocates device memory.  Errors: as
 * bs_plan_create, BS_ERR_OOM. */
bs_status bs_mc_create(const bs_plan_desc *group_descs, int ngroups, bs_mc *out);
bs_status bs_mc_destroy(bs_mc mc);
/* Message of the last failure on this ensemble; never NULL. */
const char *bs_mc_last_error(bs_mc mc);
/* bs_plan_info of group g's plan. */
bs_status bs_mc_info(bs_mc mc, int group, int64_t *info_host, int n);
/* Register group g's input: a caller-owned device buffer of complex64
 * [batch][nchan][nt][nt] visibilities, centred, Hermitian, 8-byte aligned.
 * The caller writes the next realisations there before each bs_mc_run and
 * keeps the buffer alive; registering a different pointer drops the captured
 * graph (it is captured again on the next graph run). */
bs_status bs_mc_set_input(bs_mc mc, int group, const void *vis_dev);
/* Channel flags of group g (uint8 [nchan], nonzero = flagged; NULL = none):
 * flagged channels have W = 0 (Eq. vg), so their triples are undefined and
 * the collapse and Eq. (dft) use only sampled separations.  Drops prepared
 * work and the captured graph. */
bs_status bs_mc_set_flags(bs_mc mc, int group, const uint8_t *flags_host);
/* Tuning knob chosen by the autotuner: split K until the contraction has at
 * least tiles_per_sm tiles per SM (1..64).  Only before the first run. */
bs_status bs_mc_set_tuning(bs_mc mc, int tiles_per_sm);
/* Autotuner over the tile shapes of the persistent contraction.  A tile is
 * 256 fields x 512 channel pairs (fixed by the two-SM MMA and the pair
 * producers) x a K range; the tuner chooses the K extent (split K until the
 * launch holds at least tiles_per_sm tiles per SM, tiles_per_sm in
 * {1, 2, 4, 8, 16}) and then the tile order (0: longest K first across
 * groups, 1: group and ring-pair order, which keeps neighbouring CTA pairs on
 * the same field rows).  Each candidate: one warm-up and two timed runs on the
 * registered inputs.  The choice is stored in the JSON file cache_path under
 * the ensemble's shape signature (shapes, rings, channel blocks; NULL: no
 * cache); a cached signature is applied without timing.  Resets the
 * statistics; writes the chosen tiles_per_sm to *chosen (bs_mc_tuning gives
 * both knobs).  Synchronises. */
bs_status bs_mc_autotune(bs_mc mc, const char *cache_path, int *chosen, void *cuda_stream);
/* The tuning in effect: K-split target and tile order (either pointer may be NULL). */
bs_status bs_mc_tuning(bs_mc mc, int *tiles_per_sm, int *tile_order);
/* The channel block each run of group g contracts, int32 [6] = {nu1_lo,
 * nu1_hi, nu2_lo, nu2_hi, nu3_lo, nu3_hi} (default: the full cube): a
 * declared subset of the tiles of every realisation, for ensembles whose
 * full channel cubes are too large to run (the collapse and Eq. (dft) then
 * hold the separations of that block).  A cube block of 64 channels or
 * more (the full cube included) is contracted with the channel symmetry of
 * repeated rings, as bs_mabs with accumulate = 2.  Drops prepared work and
 * the captured graph.  Errors: BS_ERR_ARG (group, NULL, block out of range
 * or empty). */
bs_status bs_mc_set_block(bs_mc mc, int group, const int32_t *block_host);
/* One Monte Carlo step over all groups (asynchronous on cuda_stream). */
bs_status bs_mc_run(bs_mc mc, int use_graph, void *cuda_stream);
/* Zero the statistics. */
bs_status bs_mc_reset(bs_mc mc, void *cuda_stream);
/* Per-bin statistics of group g over all realisations accumulated so far:
 *  which = 0: folded collapsed MABS, bins [T_r][2nchan-1][2nchan-1]
 *  which = 1: 3D bispectrum of Eq. (dft), bins [T_r][nchan][nchan]
 *  mean_dev / var_dev: double device arrays of that size (either may be
 *  NULL); var is the unbiased sample variance; NaN where fewer than 1 (mean)
 *  or 2 (var) defined values.  realisations_host (or NULL): realisations of
 *  group g accumulated.  Synchronises to read the device error word; returns
 *  BS_ERR_TIMEOUT if a bounded wait gave up. */
bs_status bs_mc_stats(bs_mc mc, int group, int which, double *mean_dev, double *var_dev,
                      int64_t *realisations_host, void *cuda_stream);

/* Checkpoint and resume of a long Monte Carlo run (not in the paper).
 * bs_mc_checkpoint synchronises on cuda_stream and writes to the file `path`
 * (written to path.tmp, then renamed): the ensemble's shape signature, the
 * per-bin Welford state (count, mean, M2) of every group, the runs so far, the
 * tuning, and `counter`, a value of the caller's -- e.g. the realisation index
 * that the next bs_sky_generate call starts at (the Philox counter), so that a
 * resumed run draws the realisations that the interrupted one would have.
 * bs_mc_restore reads such a file into an ensemble of the same shapes, returns
 * the counter, and replaces the statistics, the run count and the tuning.
 * Errors: BS_ERR_ARG (NULL path, unreadable or unwritable file, another
 * ensemble's checkpoint), BS_ERR_CUDA. */
bs_status bs_mc_checkpoint(bs_mc mc, const char *path, uint64_t counter, void *cuda_stream);
bs_status bs_mc_restore(bs_mc mc, const char *path, uint64_t *counter, void *cuda_stream);

/* ---------------------------------------------------------------------------
 * Error-bar surrogate (not in the paper, whose error bars are brute Monte
 * Carlo over 250 realisations, Section 4): a 3-layer MLP
 *   xn = (x - mu_x)/sd_x; h1 = tanh(W1 xn + b1); h2 = tanh(W2 h1 + b2);
 *   y = mu_y + sd_y (w3 . h2 + b3)
 * with BF16 weights (rounded from FP32 masters) and FP32 accumulation,
 * trained by the library's own forward, backward and Adam kernels on the
 * per-bin log variances that bs_mc_stats produces.  Monte Carlo remains the
 * fallback and the reference its error is measured against.  Flat parameter
 * vector (float):
 *   W1 [w][d] | b1 [w] | W2 [w][w] | b2 [w] | w3 [w] | b3 | mu_x [d] | sd_x [d] | mu_y | sd_y
 * ------------------------------------------------------------------------- */
#define BS_MLP_FEATURES 45
typedef struct bs_mlp_s *bs_mlp;

/* Features of every 3D-bispectrum bin (trip, a, b) of a plan, float
 * [T_r*nchan*nchan][45] on the device, rows in bs_bs3d order:
 *  0 log k1, 1 t = k2/k1, 2 mu = (k1^2+k2^2-k3^2)/(2 k1 k2) (Eq. shape), where
 *    k_n = sqrt(k_perp n^2 + k_par n^2), k_perp = 2 pi Ubar_ring / r (ring-mean
 *    |U|), k_par a = 2 pi a / (r' nchan dnu_c), k_par 3 = -k_par a - k_par b,
 *    sorted k1 >= k2 >= k3;
 *  3 flagged fraction; 4 log T(i,j,l); 5 |k_par a|; 6 |k_par b|;
 *  7..9 log k_perp of rings i, j, l; 10..41 fraction of channels flagged at
 *  each position c mod 32 of the coarse bands; 42..44 the sampling of the
 *  Eq. (dft) square under the mask: with N(d) the folded number of valid
 *  channel triples at separation d, -nchan/2 <= d1, d2 < nchan/2,
 *  42 log sum_{N>0} 1/N, 43 fraction of separations with N > 0,
 *  44 log mean_{N>0} N (0 and 0 when nothing is sampled).
 * Rows of ring triples without closed triangles are NaN.  Synchronises. */
bs_status bs_mlp_features(bs_plan plan, const uint8_t *chan_flag_host, float *feat_dev,
                          void *cuda_stream);
/* Network with d_in inputs (<= 64) and width hidden units (<= 128), Glorot
 * initialisation from a SplitMix64 stream of seed.  Allocates device memory. */
bs_status bs_mlp_create(int d_in, int width, uint64_t seed, bs_mlp *out);
bs_status bs_mlp_destroy(bs_mlp mlp);
const char *bs_mlp_last_error(bs_mlp mlp);
/* Copy the flat parameter vector (see above; n = total length) to the host
 * (set = 0) or from the host (set = 1, also resets the Adam state). */
bs_status bs_mlp_params(bs_mlp mlp, float *params_host, int64_t n, int set);
/* Input and target normalisation from data: x_dev float [n][d_in], t_dev [n]. */
bs_status bs_mlp_fit_norm(bs_mlp mlp, const float *x_dev, const float *t_dev, int n,
                          void *cuda_stream);
/* y_dev[n] = network(x_dev[n][d_in]). */
bs_status bs_mlp_forward(bs_mlp mlp, const float *x_dev, int n, float *y_dev, void *cuda_stream);
/* Kernels of the forward, backward and weight-gradient passes: kind 0 = BF16
 * tensor cores (mma.sync m16n8k16, FP32 accumulation; activations and
 * gradients split into BF16 hi + lo, weights exact in BF16), the default
 * for width 128 and d_in <= 64; kind 1 = FP32 SIMT (any shape; the checker).
 * Errors: BS_ERR_ARG (kind), BS_ERR_UNSUPPORTED (kind 0 for another shape). */
bs_status bs_mlp_set_kernels(bs_mlp mlp, int kind);
/* Full-batch loss (mean squared error on the normalised target) and its
 * gradient w.r.t. the weights and biases (first part of the flat vector),
 * copied to the host.  Synchronises. */
bs_status bs_mlp_grad(bs_mlp mlp, const float *x_dev, const float *t_dev, int n,
                      float *grad_host, float *loss_host, void *cuda_stream);
/* `steps` Adam steps (beta 0.9/0.999) on minibatches of `batch` rows drawn
 * with replacement by a counter-based hash of (seed, step, slot); loss of the
 * last minibatch to loss_host (or NULL; synchronises when given). */
bs_status bs_mlp_train(bs_mlp mlp, const float *x_dev, const float *t_dev, int n, int steps,
                       int batch, float lr, uint64_t seed, float *loss_host, void *cuda_stream);

/* ---- Monte Carlo sky generator (the validation sky of Section 4) ---------
 * Draws realisations of the non-Gaussian sky of Eq. (mb1) on the GPU and
 * writes their gridded visibilities in the layout bs_grid_load reads, so a
 * Monte Carlo ensemble (bs_mc_*) runs with no host traffic per realisation.
 * Realisation r of a generator (nt, nchan, slope, sigma, f_ng) and a seed:
 *   w[z][y][x]  unit normals: cell c = (z nt + y) nt + x is normal c mod 4 of
 *               Philox4x32-10 (Salmon et al. 2011) call q = c div 4 with
 *               counter words (q lo, q hi, r lo, r hi) and key (seed lo,
 *               seed hi); the call's outputs (o0, o1) give cells 4q, 4q+1 by
 *               Box-Muller, sqrt(-2 ln a) (cos 2 pi b, sin 2 pi b) with
 *               a = (o0 + 1/2) 2^-32, b = (o1 + 1/2) 2^-32, and (o2, o3) give
 *               cells 4q+2, 4q+3 the same way;
 *   g           IDFT3( sqrt(P) DFT3(w) ), P(k) = A |k|^slope on the periodic
 *               box (k = 2 pi (fftfreq), unit cells), P(0) = 0, A such that
 *               the mean of P over the box is sigma^2;
 *   delta       g + f_ng (g^2 - sigma^2)                        (Eq. mb1)
 *   V[z][v + nt/2][u + nt/2] = sum_{x,y} delta[z][y][x] e^{-2 pi i (ux + vy)/nt}.
 * FP32 arithmetic (FFTs, Box-Muller); a double-precision restatement of the
 * same definition agrees to ~1e-6 of max |V|.
 *  nt         even, 8..4096;  nchan 1..4096;  both of the form 2^a 3^b 5^c
 *             (otherwise BS_ERR_UNSUPPORTED)
 *  max_batch  1..131070 realisations per bs_sky_generate call; the generator
 *             holds ceil(max_batch/2) nchan nt^2 complex64 of scratch plus a
 *             float sqrt(P) table of nchan nt^2
 * Errors: BS_ERR_ARG, BS_ERR_UNSUPPORTED, BS_ERR_NO_DEVICE, BS_ERR_OOM,
 * BS_ERR_CUDA.  bs_sky_last_error(NULL) returns the last creation error of
 * the calling thread. */
typedef struct bs_sky_s *bs_sky;
bs_status bs_sky_create(int nt, int nchan, double slope, double sigma, double f_ng, int max_batch,
                        bs_sky *out);
bs_status bs_sky_destroy(bs_sky sky);
const char *bs_sky_last_error(bs_sky sky);
/* Realisations realisation0 .. realisation0 + batch - 1 into vis_dev,
 * complex64 [batch][nchan][nt][nt] (device, caller-owned, 8-byte aligned),
 * asynchronously on cuda_stream.  Calls on one generator must not overlap on
 * the GPU (they share its scratch): use one stream per generator.
 * Errors: BS_ERR_ARG (batch outside 1..max_batch, NULL buffer), BS_ERR_STATE
 * (an earlier CUDA error), BS_ERR_CUDA. */
bs_status bs_sky_generate(bs_sky sky, uint64_t seed, uint64_t realisation0, int batch,
                          void *vis_dev, void *cuda_stream);

/* Arithmetic ceiling of the current device for roofline fractions (the paper
 * has no counterpart): kind 0 FP32 FMA, kind 1 FP64 FMA.  Every thread of
 * 4 x 256-thread blocks per SM runs 8 independent FMA chains for `iters`
 * steps on registers; *flops_per_s = 2 x FMAs / the launch's CUDA-event time
 * on cuda_stream (after one short warm-up launch).  Synchronises.
 * Errors: BS_ERR_ARG (kind, iters < 1, NULL), BS_ERR_NO_DEVICE, BS_ERR_CUDA. */
bs_status bs_measure_peak(int kind, int iters, double *flops_per_s, void *cuda_stream);

/* Closed-triangle counts T(i,j,l) without any device allocation.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc (a pipeline bound to its own pre-allocated memory
 * pool, or a host that must not touch the CUDA allocator while it shares the
 * device).  It computes the same counts as bs_counts -- ordered closed
 * triangles U_g1 + U_g2 + U_g3 = 0 with U_gk in the listed rings, empty cells
 * excluded -- with no plan: its scratch (ring labels, binned-cell list,
 * ring-triple table) is a fixed static device array of 5,374,208 bytes that
 * every device loading libbs holds until the process exits.
 *  nt              uv grid side, even, 8..1024 (larger: BS_ERR_ARG)
 *  nbins           rings, 1..32 (larger: BS_ERR_ARG)
 *  bin_edges_host  nbins+1 strictly ascending edges (|U| grid units)
 *  ngrid_dev       float [nt][nt] or NULL, as in bs_grid_load
 *  tri_dev         int64 [nbins(nbins+1)(nbins+2)/6] device output, ring
 *                  triples i <= j <= l in lexicographic order; overwritten
 * Runs on the current device, asynchronously on cuda_stream.  The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress) and,
 * under CUDA's lazy module loading, is also the call that reserves the array
 * on that device: make it (a warm-up call) before any stream capture and
 * before relying on device memory staying unchanged.  A reset of the device's
 * context frees the array; the next call notices the new context and looks
 * the address up again (reserving the array anew).  The array is shared by
 * all calls and keeps the last call's contents (the call clears what must
 * start at zero): calls that overlap on the GPU, from any stream or thread,
 * race and must be serialised by the caller.
 * Errors: BS_ERR_ARG, BS_ERR_NO_DEVICE, BS_ERR_CUDA. */
bs_status bs_counts_noalloc(int nt, int nbins, const double *bin_edges_host,
                            const float *ngrid_dev, int64_t *tri_dev, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* BS_H_ */
