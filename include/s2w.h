/*
 * s2w.h -- C ABI of the GB300 directional wavelet transform library (libs2w.so).
 *
 * The library computes the scale-discretised directional wavelet transform on the
 * sphere (Sec. 3.1 and Algorithm 1 of "Differentiable and accelerated directional
 * wavelet transforms on the sphere and ball", Price et al. 2024) on McEwen-Wiaux
 * (MW) or Driscoll-Healy (DH) sampling (the transforms are sampling agnostic, Sec. 1),
 * together with the harmonic transforms it is built from: the spin
 * spherical-harmonic transform Y (Sec. 2.1, Eqs. 2-3) and the Wigner transform D
 * (Sec. 2.2, Eqs. 4-5), and the Fourier-Laguerre radial transform of the ball
 * (Sec. 2.3, Eqs. 6-8).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Ownership   Every data pointer is a DEVICE pointer owned by the caller unless an
 *             argument says otherwise.  A plan owns its tables and a workspace
 *             sized for its batch; execute calls allocate nothing and do not
 *             synchronise the host, so they can be issued back to back on a stream.
 * Streams     `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *             stream).  All work of a call is enqueued on that stream; calls that
 *             share one plan must not run concurrently (they share its workspace).
 * Elements    float64.  A plan with reality=1 and spin=0 takes and returns REAL
 *             pixel arrays (double); otherwise pixel arrays are complex,
 *             interleaved (re, im) pairs of double.  Harmonic-space arrays are
 *             always complex interleaved.
 * Sampling    R(L) colatitude rings by 2L-1 longitudes phi_p = 2 pi p/(2L-1) at band-limit L:
 *             MW  R = L rings theta_t = pi(2t+1)/(2L-1), t < L (the last is the south pole);
 *             DH  R = 2L rings theta_t = pi(2t+1)/(4L), t < 2L (no pole sampled).
 *             On SO(3) beta takes the theta rings and alpha the phi samples.
 * Layouts     (row-major, batch outermost; `b` = batch index)
 *   map       [b][R(L) theta][2L-1 phi]
 *   wav       scales j = J0..J concatenated; scale j is [b][2N_j-1 gamma][R(L_j) beta][2L_j-1 alpha]
 *             with gamma_g = 2 pi g/(2N_j-1) and alpha, beta on the grid at L_j
 *   scal      [b][R(L_Phi)][2L_Phi-1] (the grid at the scaling band-limit L_Phi)
 *   flm       [b][L][Mc] with Mc = L (m = 0..L-1) for real plans and Mc = 2L-1
 *             (index m + L - 1) otherwise; real signals obey f_{l,-m} = (-1)^m conj f_lm
 *   flmn      [b][2N_j-1][L_j][Mc_j], n index n + N_j - 1, m indexed as for flm at L_j
 * Errors      Every call returns an s2w_status.  Parameters are validated at plan
 *             creation and on each call (null or misaligned pointers, bad scale
 *             index).  s2w_last_error() returns a thread-local message for the most
 *             recent failure.  Device-side problems are recorded in a per-plan error
 *             word that s2w_check() reads; nothing traps or aborts.
 */
#ifndef S2W_H
#define S2W_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  S2W_OK = 0,
  S2W_EINVAL = 1,        /* bad parameter or pointer */
  S2W_ENOMEM = 2,        /* device allocation failed at plan creation */
  S2W_ECUDA = 3,         /* a CUDA runtime call or kernel launch failed */
  S2W_ETIMEOUT = 4,      /* a bounded device wait gave up */
  S2W_EUNSUPPORTED = 5,  /* parameters valid but not supported by this build */
  S2W_ENONFINITE = 6     /* a kernel detected a non-finite input */
} s2w_status;

/* S2W_FP64         float64 accuracy (1e-11 target): Wigner-d recursion and l-contractions in
 *                  float64; DFTs in compensated float32 pairs (error-free transformations).
 * S2W_FP64_NATIVE  every step in native float64: the plain float64 path, kept as the
 *                  baseline the other modes are compared with.
 * S2W_FP32_SPLIT  wavelet-scale l-contractions on the tensor cores (tcgen05) against
 *                  precomputed Wigner-d tables stored as fp16 hi + lo pairs, data as fp16
 *                  pairs, float32 accumulation (1e-5 target); plain float32 DFTs there.
 * S2W_BF16         split-bf16: the same with bf16 hi + lo pairs for the tables and the data
 *                  (the products hi*hi, hi*lo, lo*hi per K step, float32 accumulation; 1e-3
 *                  target).
 *                  Both reduced modes keep the spin SHT Y, Y^-1 and the scaling transform
 *                  float64-accurate (on the sliced tensor-core kernels of S2W_FP64_TC) and
 *                  support L and the ring count <= 512 (S2W_EUNSUPPORTED above).
 * S2W_FP64_TC      float64 accuracy (1e-11 target) with every l-contraction on the tensor cores:
 *                  precomputed Wigner-d tables and the data cut into seven 7-bit integer slices
 *                  (bf16), the slice products exact and their float32 sums exact (Ozaki's
 *                  error-free splitting); the azimuthal DFTs on the tensor cores by the same
 *                  slicing: the prime-factor form (2L - 1 = n1 n2, the n2-point stage a sliced
 *                  GEMM, the n1-point stage and the gamma DFT in compensated float32) where
 *                  2L - 1 factors with n2 < 128, else the direct form (the symmetric odd-length
 *                  DFT as two GEMMs against sliced twiddle tables) where the carried n fit (at
 *                  most 16 per ring), else compensated float32 pairs; s2w_plan_autotune picks
 *                  among them by timing, s2w_plan_set_dft_forms forces one.  The tables are
 *                  always precomputed (precompute is ignored).  L <= 512 and at most 512 rings
 *                  (S2W_EUNSUPPORTED above). */
typedef enum { S2W_FP64 = 0, S2W_FP32_SPLIT = 1, S2W_BF16 = 2, S2W_FP64_NATIVE = 3, S2W_FP64_TC = 4 } s2w_precision;

/* S2W_SAMPLING_MW  McEwen-Wiaux: L rings; the forward transforms' colatitude integral is
 *                  exact through the periodic extension of each column (a dense quadrature
 *                  matrix per parity of m + n).
 * S2W_SAMPLING_DH  Driscoll-Healy: 2L midpoint rings; the colatitude integral is the
 *                  weighted ring sum with the weights w_t that integrate cos(k theta) sin(theta)
 *                  exactly for k < 2L (Fejer's first rule in x = cos theta).  L <= 512. */
typedef enum { S2W_SAMPLING_MW = 0, S2W_SAMPLING_DH = 1 } s2w_sampling;

/* Problem statement of the sphere transform (Algorithm 1; Sec. 3.3; App. A).
 *   L        angular band-limit, harmonic degrees l < L            (2 <= L <= 1024)
 *   N        azimuthal band-limit of the wavelets, |n| < N          (1 <= N <= L)
 *   J0       lowest wavelet scale; the scaling function covers l < lambda^J0
 *   spin     spin of the signal, |spin| < L
 *   reality  1 for real spin-0 signals (real pixel arrays, m >= 0 stored)
 *   batch    number of maps transformed per call                   (>= 1)
 *   precision  s2w_precision
 *   precompute 0 (Wigner-d functions by recursion inside the kernels)
 *   lambda   dilation factor lambda > 1 (Eq. A2); scale j uses band-limit
 *            L_j = min(ceil(lambda^(j+1)), L) and N_j = min(N, L_j), j = J0..J with J
 *            the smallest integer such that lambda^J >= L; L_Phi = min(ceil(lambda^J0), L).
 *   sampling s2w_sampling (0 = MW, the default of a zeroed struct) */
typedef struct {
  int L, N, J0, spin, reality, batch, precision, precompute;
  double lambda;
  int sampling;
} s2w_params;

typedef struct s2w_plan s2w_plan;

/* Builds every table the transforms need (filters, quadrature matrices, Wigner-d
 * seeds, DFT twiddles) in float64 on the host, uploads them and allocates the
 * workspace.  Blocks until the uploads are complete.  *out receives the plan;
 * on failure *out is NULL and nothing is leaked.  `stream` is only used for the
 * uploads. */
s2w_status s2w_plan_create(const s2w_params* params, void* stream, s2w_plan** out);

/* Frees the plan.  The caller must make sure no work using it is still queued. */
s2w_status s2w_plan_destroy(s2w_plan* plan);

/* Device memory the plan holds, in bytes (HOST pointers, either may be NULL): *table_bytes its
 * precomputed tables (Wigner-d tables of the precomputed modes, as in the paper's precompute mode
 * of Sec. 4.2, quadrature matrices, twiddles, seeds, filters); *workspace_bytes the per-call
 * scratch sized for its batch (columns, harmonic workspace, data slices).  Temporary tables freed
 * during plan creation are not counted. */
s2w_status s2w_plan_device_bytes(const s2w_plan* plan, int64_t* table_bytes, int64_t* workspace_bytes);

/* Sizes (in elements of the plan's pixel type, per map) of the map, the
 * concatenated wavelet coefficients and the scaling coefficients; the number of
 * scales; wav_offsets[0..nscales] (element offsets of each scale inside one map's
 * wavelet block, last = total); and per scale L_j, N_j.  Any output pointer may be
 * NULL.  Arrays must hold nscales (+1 for offsets) entries; query nscales first with
 * the others NULL.  *L_phi receives the scaling band-limit. */
s2w_status s2w_query_layout(const s2w_plan* plan, int64_t* map_elems, int64_t* wav_elems,
                            int64_t* scal_elems, int* nscales, int64_t* wav_offsets,
                            int* Lj, int* Nj, int* L_phi);

/* Analysis (Algorithm 1, Eqs. 40-41): f [batch][map] -> wav, scal. */
s2w_status s2w_forward(const s2w_plan* plan, const void* f, void* wav, void* scal, void* stream);

/* Synthesis (Algorithm 1, Eq. 42): wav, scal -> f.  Exact inverse of s2w_forward on
 * band-limited signals (the admissibility condition, Eq. 30). */
s2w_status s2w_inverse(const s2w_plan* plan, const void* wav, const void* scal, void* f,
                       void* stream);

/* ---- adjoints (Sec. 4.3: the transforms are differentiable; the gradient of a loss
 * through a linear transform is its adjoint applied to the loss's gradient) -------------
 * Both are linear maps between the same buffers as the transforms they transpose, with
 * the roles of input and output exchanged; layouts and element types as above.  The adjoint
 * is taken for the inner product <x, y> = Re sum conj(x_i) y_i over every stored sample;
 * for real plans (real maps and real wavelet coefficients) that is the ordinary transpose.
 * Every step of the transform is transposed in order: the DFTs (forward <-> inverse with
 * the normalisation moved), the l-contraction (the same recursion, summed over the other
 * index), the harmonic products (conjugated) and the colatitude quadrature (its transpose,
 * applied between the inverse contraction and the inverse DFT).  The Wigner-d values are
 * recomputed by the recursion, never stored.  Accuracy: float64 (<= 1e-11 relative) in
 * every precision mode; the reduced modes run their adjoints on the float64-accurate
 * kernels.  Same stream, allocation and error behaviour as s2w_forward. */

/* Adjoint of s2w_forward: (gwav, gscal) -> gf.  gf = A^H (gwav, gscal) where A is the
 * analysis operator f -> (wav, scal) of Eqs. 40-41.  gf is overwritten. */
s2w_status s2w_forward_adjoint(const s2w_plan* plan, const void* gwav, const void* gscal, void* gf,
                               void* stream);

/* Adjoint of s2w_inverse: gf -> (gwav, gscal).  (gwav, gscal) = S^H gf where S is the
 * synthesis operator (wav, scal) -> f of Eq. 42.  gwav and gscal are overwritten. */
s2w_status s2w_inverse_adjoint(const s2w_plan* plan, const void* gf, void* gwav, void* gscal,
                               void* stream);

/* Forward spin SHT (Eq. 2) of the plan's batch of maps at band-limit L and spin: f -> flm. */
s2w_status s2w_sht_forward(const s2w_plan* plan, const void* f, void* flm, void* stream);

/* Inverse spin SHT (Eq. 3): flm -> f. */
s2w_status s2w_sht_inverse(const s2w_plan* plan, const void* flm, void* f, void* stream);

/* Forward Wigner transform (Eq. 4) at the band-limits (L_j, N_j) of wavelet scale
 * index `scale` (0 = J0): SO(3) samples laid out like one scale of `wav` -> flmn
 * (all |n| < N_j, layout above). */
s2w_status s2w_wigner_forward(const s2w_plan* plan, int scale, const void* f, void* flmn,
                              void* stream);

/* Inverse Wigner transform (Eq. 5) at (L_j, N_j): flmn -> SO(3) samples. */
s2w_status s2w_wigner_inverse(const s2w_plan* plan, int scale, const void* flmn, void* f,
                              void* stream);

/* ---- ball: Fourier-Laguerre radial transform and spherical-Laguerre transform ----------
 * (Sec. 2.3, Eqs. 6-11.)  Radial basis K_p(r) = sqrt(p!/(p+2)!) e^{-r/(2 tau)} tau^{-3/2}
 * L^(2)_p(r/tau) (Eq. 6), radial band-limit p < P.  The radial samples are the P generalised
 * Gauss-Laguerre nodes r_i = tau x_i (roots of L^(2)_P) with weights omega_i such that the
 * forward transform f_p = sum_i omega_i K_p(r_i) f(r_i) (Eq. 7) is exact for band-limited
 * signals; the inverse is f(r_i) = sum_p K_p(r_i) f_p (Eq. 8).
 * Layouts (b = batch index): radial samples of harmonic coefficients f_r [b][P node][L][Mc] and
 * Fourier-Laguerre coefficients f_p [b][P][L][Mc], complex; ball pixels [b][P node][R(L)][2L-1]
 * on the angular sampling `sampling` (real when reality = 1, else complex).  The plan owns a
 * workspace of batch*P*L*Mc complex. */
typedef struct {
  int L;          /* angular band-limit (2 <= L <= 1024) */
  int P;          /* radial band-limit (2 <= P <= 256) */
  int spin, reality, batch, precision;   /* as in s2w_params; in the tensor-core modes (S2W_FP32_SPLIT,
                                            S2W_BF16, S2W_FP64_TC) the radial maps run on the tensor
                                            cores as exact sliced GEMMs (float64-accurate) */
  double tau;     /* Laguerre scale tau > 0 */
  int sampling;   /* angular sampling, s2w_sampling */
} s2w_ball_params;

typedef struct s2w_ball_plan s2w_ball_plan;

/* Builds the radial quadrature and matrices in float64 on the host (sliced for the tensor cores in
 * the tensor-core modes) and an SHT plan for batch*P maps; blocks until uploads complete. */
s2w_status s2w_ball_plan_create(const s2w_ball_params* params, void* stream, s2w_ball_plan** out);
s2w_status s2w_ball_plan_destroy(s2w_ball_plan* plan);
/* Copies the nodes r_i and weights omega_i (P doubles each, HOST pointers, may be NULL). */
s2w_status s2w_ball_nodes(const s2w_ball_plan* plan, double* r, double* omega);
/* Eq. 7 on every angular coefficient column: f_r -> f_p. */
s2w_status s2w_laguerre_forward(const s2w_ball_plan* plan, const void* f_r, void* f_p, void* stream);
/* Eq. 8: f_p -> f_r. */
s2w_status s2w_laguerre_inverse(const s2w_ball_plan* plan, const void* f_p, void* f_r, void* stream);
/* Z (Eq. 10): ball pixels -> f_lmp = Laguerre-forward of the per-node spin SHT. */
s2w_status s2w_ball_sl_forward(const s2w_ball_plan* plan, const void* f, void* flmp, void* stream);
/* Z^-1 (Eq. 11): f_lmp -> ball pixels. */
s2w_status s2w_ball_sl_inverse(const s2w_ball_plan* plan, const void* flmp, void* f, void* stream);

/* ---- ball: directional wavelet transform (Sec. 3.2; Sec. 5.1, Algorithm 2) ----------------
 * Wavelets Psi^{jj'}_lnp = sqrt((2l+1)/(8 pi^2)) kappa^j(l) kappa^{j'}(p) zeta_ln (App. A.4) for
 * angular scales j = J0..J (as in s2w_params) and radial scales j' = J0r..J', J' the smallest
 * integer with nu^J' >= P, kappa^{j'}(p) = kappa_nu(p / nu^j').  Multiresolution (Sec. 3.3):
 * scale (j, j') is sampled on the SO(3) grid of the sampling at (L_j, N_j) and on the P_j'-node
 * Gauss-Laguerre rule, P_j' = min(ceil(nu^(j'+1)), P), r'_i = tau x'_i.  Scaling function:
 * |Phi_l0p|^2 (4 pi/(2l+1)) = A + B - A B with A = k_lambda(l/lambda^J0), B = k_nu(p/nu^J0r)
 * (the reading of App. A.4 that satisfies the admissibility condition of Sec. 3.2); the
 * scaling coefficients W^Phi are sampled at full resolution (P nodes, the grid at L).
 * Spin 0 only (S2W_EUNSUPPORTED otherwise); real fields when reality = 1.
 * Layouts: field f and scaling coefficients [batch][P node][R(L)][2L-1]; wavelet coefficients
 * wav: one block per scale k in the order of s2w_ball_wav_query_layout (j outer, j' inner),
 * block k = [batch][P_j' node][2N_j-1 gamma][R(L_j) beta][2L_j-1 alpha], starting at element
 * wav_offsets[k] (offsets over the WHOLE batch, unlike s2w_query_layout).
 * The plan holds a sphere wavelet plan over batch*P node maps and two workspaces of
 * batch*P*L*Mc complex.  Every precision mode is accepted: the sphere transforms run in it, and in
 * the tensor-core modes (S2W_FP32_SPLIT, S2W_BF16, S2W_FP64_TC) every radial map (the
 * Fourier-Laguerre transform, its inverse, the per-scale filters and their transposes) runs on the
 * tensor cores as an exact sliced GEMM, float64-accurate.  Same stream, allocation and error
 * conventions as s2w_forward. */
typedef struct {
  int L, N, P, J0, J0r, spin, reality, batch, precision, precompute;   /* precision/precompute as s2w_params */
  double lambda, nu, tau;
  int sampling;   /* angular sampling, s2w_sampling */
} s2w_ball_wav_params;

typedef struct s2w_ball_wav_plan s2w_ball_wav_plan;

s2w_status s2w_ball_wav_plan_create(const s2w_ball_wav_params* params, void* stream, s2w_ball_wav_plan** out);
s2w_status s2w_ball_wav_plan_destroy(s2w_ball_wav_plan* plan);
/* Element counts of one field and of all wavelet blocks; the number of scales; per scale k its
 * (j, j'), offset, L_j, N_j and P_j' (arrays of nscales entries, offsets nscales+1; any may be
 * NULL; query nscales first). */
s2w_status s2w_ball_wav_query_layout(const s2w_ball_wav_plan* plan, int64_t* field_elems, int64_t* wav_elems,
                                     int* nscales, int* j, int* jr, int64_t* wav_offsets, int* Lj, int* Nj,
                                     int* Pj);
/* Analysis (Sec. 5.1, Algorithm 2): f -> wav, scal. */
s2w_status s2w_ball_forward(const s2w_ball_wav_plan* plan, const void* f, void* wav, void* scal, void* stream);
/* Synthesis (Sec. 5.1, Eq. for the inverse): wav, scal -> f; exact inverse of s2w_ball_forward on
 * band-limited fields. */
s2w_status s2w_ball_inverse(const s2w_ball_wav_plan* plan, const void* wav, const void* scal, void* f,
                            void* stream);
/* Adjoints (transposes for real fields) of the two, as for the sphere. */
s2w_status s2w_ball_forward_adjoint(const s2w_ball_wav_plan* plan, const void* gwav, const void* gscal, void* gf,
                                    void* stream);
s2w_status s2w_ball_inverse_adjoint(const s2w_ball_wav_plan* plan, const void* gf, void* gwav, void* gscal,
                                    void* stream);
/* s2w_check of the plan's sphere transforms (synchronises, reads the device error word). */
s2w_status s2w_ball_wav_check(const s2w_ball_wav_plan* plan);
/* s2w_plan_autotune on the plan's sphere transforms (the batch of B P node maps): launch shapes
 * and, in S2W_FP64_TC, the DFT form of each transform and direction.  Same contract as
 * s2w_plan_autotune (synchronises, overwrites the workspaces); the paper has no counterpart. */
s2w_status s2w_ball_wav_plan_autotune(s2w_ball_wav_plan* plan, void* stream);

/* The inverse spin SHT of s2w_sht_inverse, for callers that cannot allocate device memory
 * when they need it (a host application that owns every device allocation and forbids new
 * ones after start-up, or code running while a CUDA graph is captured, where cudaMalloc is not
 * allowed) and cannot borrow the plan's workspace because another call on the same plan may be
 * running.  The paper has no counterpart.
 * Its m-column scratch is a fixed 16 MiB device array inside the library (held by every GPU
 * that loads it, until exit): the call allocates nothing and returns S2W_EINVAL when
 * batch * R(L) * Mc exceeds 1,048,576 complex elements (R(L) = L rings on MW, 2L on DH; e.g. 16
 * real MW maps at L = 256).  Every call made outside stream capture looks the array's device
 * address up and caches it per device; a call made during capture uses the cached address, so
 * make one call on each device before capturing (and again after cudaDeviceReset).  All calls
 * share the array and it keeps the previous call's contents (every element a call reads it has
 * written first); calls whose work overlaps on the GPU race on it.  Same arguments and layouts as
 * s2w_sht_inverse; the l-contraction always runs the on-the-fly Wigner-d recursion (whatever the
 * plan's precision mode), so the results match s2w_sht_inverse to the float64 tolerance (1e-11
 * relative), not bit for bit. */
s2w_status s2w_sht_inverse_static(const s2w_plan* plan, const void* flm, void* f, void* stream);

/* ---- m-sharded spin SHT (Sec. 4.3: one transform spread over several GPUs) ----------------
 * The spin SHT factors into an l-contraction that is independent for every azimuthal frequency m
 * (the sum over l of Eq. 3 at fixed m; for the forward transform, Eq. 2, with the colatitude
 * quadrature of each m column, Sec. 3.2) and an azimuthal DFT that is independent for every
 * colatitude ring.  These stage calls run each part on a range of m columns or of rings, so that
 * R ranks can split one transform: rank r contracts its columns, the ranks exchange one block of
 * the column buffer each (an all-to-all: rank r sends the rows of rank q's rings and its own
 * columns to rank q), and rank r transforms its rings; the forward direction runs the same steps
 * in the opposite order.  The paper distributes its transforms over GPUs without naming the
 * index it splits; the order m is the reading taken here.
 *
 * Column buffer cols: [batch][R(L)][Mc] complex float64 (R(L) = L rings on MW, 2L on DH; Mc = L
 * columns m = 0..L-1 for real maps, else 2L-1 columns m = -(L-1)..L-1), column c holding
 * m = c + m_min, row t ring t.  A contraction call reads or writes only columns [c_begin, c_end)
 * of cols, a DFT call only rows [ring_begin, ring_end); ranges need 0 <= begin <= end <= Mc or
 * R(L) (S2W_EINVAL otherwise), and an empty range does nothing.  Every stage runs the
 * float64-accurate on-the-fly path in every precision mode (the Wigner-d recursion of S2W_FP64
 * and compensated float32 DFTs; native float64 in S2W_FP64_NATIVE), so the stages composed over
 * all ranges match s2w_sht_forward / s2w_sht_inverse to the float64 tolerance (1e-11 relative).
 * flm and f have the layouts of s2w_sht_forward / s2w_sht_inverse.
 *
 * s2w_shard_layout: the ranges of rank `rank` of `nranks` for a plan with band-limit L, spin,
 * reality and sampling (host only: no plan, no GPU).  Columns are split into contiguous ranges of
 * near-equal contraction work (column m costs L - max(|m|, |spin|) degrees l), rings into
 * contiguous ranges of near-equal count (floor(r R(L) / nranks) .. floor((r + 1) R(L) / nranks)).
 * A rank may get an empty range when nranks exceeds the columns or rings. */
s2w_status s2w_shard_layout(int L, int spin, int reality, int sampling, int nranks, int rank, int* c_begin,
                            int* c_end, int* ring_begin, int* ring_end);
/* flm -> columns [c_begin, c_end) of cols (every ring). */
s2w_status s2w_sht_inverse_columns(const s2w_plan* plan, const void* flm, void* cols, int c_begin, int c_end,
                                   void* stream);
/* rows [ring_begin, ring_end) of cols (every column) -> those rings of f; other rings untouched. */
s2w_status s2w_sht_inverse_rings(const s2w_plan* plan, const void* cols, void* f, int ring_begin, int ring_end,
                                 void* stream);
/* rings [ring_begin, ring_end) of f -> rows [ring_begin, ring_end) of cols (every column). */
s2w_status s2w_sht_forward_rings(const s2w_plan* plan, const void* f, void* cols, int ring_begin, int ring_end,
                                 void* stream);
/* columns [c_begin, c_end) of cols (every ring) -> the coefficients of those m in flm (every l,
 * overwritten); other m untouched. */
s2w_status s2w_sht_forward_columns(const s2w_plan* plan, const void* cols, void* flm, int c_begin, int c_end,
                                   void* stream);

/* ---- runtime: autotuner and batch executor ------------------------------------------
 * s2w_plan_autotune times, on the plan's own shapes and workspace, the candidate launch shapes
 * of its kernels (threads per block of the DFT kernels: 128, 256, 384, 512; maps per block of the
 * on-the-fly inverse contraction: 4, 8, 16) for every transform of the plan (spin SHT,
 * scaling function, each wavelet scale) and keeps the fastest.  In S2W_FP64_TC it also times
 * the forms of the azimuthal DFTs of each transform and direction (tensor-core prime-factor,
 * tensor-core direct, compensated float32; all float64-accurate) and keeps the fastest; without
 * autotuning the prime-factor form runs wherever its tables exist, else the direct form.
 * Synchronises the stream; allocates a pixel scratch for the
 * duration of the call; overwrites the plan's workspaces.  The paper has no counterpart (its
 * kernels are compiled by XLA). */
s2w_status s2w_plan_autotune(s2w_plan* plan, void* stream);
/* The launch shapes in use for transform `transform` (0 = spin SHT, 1 = scaling function,
 * 2 + s = wavelet scale s); any output may be NULL. */
s2w_status s2w_plan_launch_shapes(const s2w_plan* plan, int transform, int* dft_threads_fwd,
                                  int* dft_threads_inv, int* inv_mb);
/* The form of the azimuthal DFTs in use for transform `transform` (numbering as above), forward
 * and inverse: 2 = tensor cores, prime-factor form (S2W_FP64_TC where 2L-1 = n1 n2 fits the
 * kernel: the n2-point stage an exact sliced GEMM against a table resident in shared memory, the
 * n1-point stage and the gamma DFT in compensated float32, one persistent kernel per direction;
 * the default wherever its tables exist), 1 = tensor cores, direct form (the symmetric
 * odd-length DFT as two sliced GEMMs streaming their twiddle tables), 0 = the precision mode's
 * SIMT kernels; either output may be NULL.  The paper has no counterpart. */
s2w_status s2w_plan_dft_forms(const s2w_plan* plan, int transform, int* tc_fwd, int* tc_inv);
/* Forces the forms of transform `transform`'s azimuthal DFTs (codes as above, -1 = the default);
 * S2W_EUNSUPPORTED if the plan has no tables for a requested tensor-core form (every form is
 * float64-accurate, so results agree to the float64 tolerance).  For tests and comparisons; the
 * paper has no counterpart. */
s2w_status s2w_plan_set_dft_forms(s2w_plan* plan, int transform, int fwd, int inv);

/* A batch runs the transforms of `count` distinct plans (maps of different band-limits, spins
 * and sizes) as one CUDA graph: the plans' calls are captured once on a fork of streams (one
 * per plan), so independent transforms overlap on the GPU, and s2w_batch_launch replays the
 * whole graph with one launch.  what = 0: analysis in[i] -> wav[i], scal[i]; 1: synthesis
 * wav[i], scal[i] -> out[i]; 2: both in sequence.  The device buffers are fixed at creation
 * (arrays of count pointers; in or out may be NULL when unused) and must outlive the batch.
 * A plan may appear once.  The plans must not be used by other calls while a launch of the
 * batch is running (they share the plans' workspaces).  (Batching of Sec. 4.3; the graph is
 * this library's form of it.) */
typedef struct s2w_batch s2w_batch;
s2w_status s2w_batch_create(s2w_plan* const* plans, int count, const void* const* in, void* const* wav,
                            void* const* scal, void* const* out, int what, void* stream, s2w_batch** batch);
s2w_status s2w_batch_launch(s2w_batch* batch, void* stream);
s2w_status s2w_batch_destroy(s2w_batch* batch);

/* Synchronises the plan's last stream, then reads and clears the device error word.
 * Returns S2W_OK, S2W_ECUDA (asynchronous CUDA error) or the recorded status:
 *   S2W_ETIMEOUT    a bounded mbarrier wait of a tensor-core kernel ran out (the kernel set the
 *                   word, let its own copies and MMAs in flight land, freed its tensor memory and
 *                   returned; the outputs of that call are undefined, the context stays usable);
 *   S2W_ENONFINITE  S2W_FP64_TC (and the reduced modes' SHT and scaling transform, which run
 *                   on its kernels): the exponent pass that reads every value before the
 *                   tensor-core slicing met a NaN or Inf (in the input, or produced from it), so
 *                   the outputs of that call are not meaningful.  The other modes do not check and
 *                   propagate NaN and Inf to the outputs. */
s2w_status s2w_check(const s2w_plan* plan);

/* Failure-path test hook (the paper has no counterpart): while on != 0, every tensor-core
 * l-contraction launch of the plan (S2W_FP64_TC) makes its first bounded mbarrier wait wait on a
 * barrier that nothing completes, so the wait runs out after its poll limit with bulk copies in
 * flight and the kernel takes its timeout path; s2w_check then returns S2W_ETIMEOUT.  No fault,
 * trap or hang is involved.  on = 0 restores normal operation. */
s2w_status s2w_plan_inject_timeout(s2w_plan* plan, int on);

/* Message for the most recent failing call on this thread ("" if none). */
const char* s2w_last_error(void);

/* Library version string. */
const char* s2w_version(void);

/* ---- tracing ------------------------------------------------------------------------
 * Kernel kinds reported by the tracer:
 *   0 "dft_forward"   pixels -> m-columns (azimuthal + gamma DFTs)
 *   1 "dft_inverse"   m-columns -> pixels
 *   2 "wigner_inverse" inverse l-contraction with the fused Wigner-d recursion
 *   3 "wigner_forward" colatitude quadrature + forward l-contraction
 *   4 "quadrature_adjoint" transposed colatitude quadrature (adjoints only)
 * When tracing is on, every kernel launch of the plan is bracketed by two CUDA events
 * recorded on the launching stream (events come from a pool created by
 * s2w_trace_enable; launches beyond its capacity are not recorded).  Besides the device
 * time, the tracer accumulates each launch's ALGORITHMIC float64 operation count:
 *   dft_*      2.5 n log2 n per real ring transform of length n (half a complex FFT) plus
 *              8 per gamma-DFT multiply-add;
 *   wigner_*   per contraction term (beta, m, n, l >= max|m|,|n|): 5 for the recursion
 *              step plus 4 per map (complex coefficient times real d^l_mn);
 *              the dense colatitude quadrature of wigner_forward is not counted;
 *   quadrature_adjoint  4 per (map, n, m, t, t') (complex column times real matrix):
 *              the transposed quadrature has no cheaper form in this design, so its dense
 *              cost is the count. */
s2w_status s2w_trace_enable(s2w_plan* plan, int on, int capacity);
/* Clears the recorded launches (does not synchronise). */
s2w_status s2w_trace_reset(s2w_plan* plan);
/* Synchronises the recorded events and returns, for kernel kind `kind`, the number of
 * recorded launches, their summed device time in milliseconds and summed algorithmic
 * float64 operations.  Any output pointer may be NULL. */
s2w_status s2w_trace_read(const s2w_plan* plan, int kind, int64_t* launches, double* ms,
                          double* flops);
/* Name of a kernel kind ("" if out of range). */
const char* s2w_kernel_name(int kind);

#ifdef __cplusplus
}
#endif

#endif /* S2W_H */
