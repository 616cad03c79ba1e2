// Internal structures shared by the host plan builder and the CUDA kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/s2w.h"

namespace s2w {

// Number of colatitude rings of the grid at band-limit L: L on McEwen-Wiaux sampling
// (theta_t = pi (2t+1)/(2L-1)), 2L on Driscoll-Healy sampling (theta_t = pi (2t+1)/(4L)).
inline int rings_of(int sampling, int L) { return sampling == S2W_SAMPLING_DH ? 2 * L : L; }

// Tables for one band-limit L on the plan's sampling (shared by every transform run at that
// L).  Device pointers; rows are padded to the row lengths given.
struct GridTables {
  int L = 0;            // band-limit (n = 2L-1 azimuthal samples)
  int nr = 0;           // colatitude rings: L (MW) or 2L (DH)
  int den = 0;          // ring t sits at theta_t = pi (2t+1)/den: den = 2L-1 (MW) or 4L (DH)
  int n = 0;            // 2L-1
  int n1 = 1, n2 = 1;   // DFT factorisation n = n1 * n2 (n1 = 1 for primes)
  double* wpole = nullptr;     // [nr] -2 sin^2(beta_b/2) (beta < pi/2) or 2 cos^2(beta_b/2) (beta >= pi/2)
  double* cpow_m = nullptr;    // [nr][n] mantissa of cos(beta_b/2)^a, a = 0..n-1
  int* cpow_e = nullptr;       // [nr][n] binary exponent
  double* spow_m = nullptr;    // [nr][n] sin(beta_b/2)^a
  int* spow_e = nullptr;
  double* sqrtC = nullptr;     // [L][n] sqrt(binom(2l, k)), k = 0..2l
  // colatitude quadrature of the forward transforms: MW has a dense matrix per parity of
  // m + n, DH a diagonal (the ring weights), the same for both parities
  double* MT = nullptr;        // MW: [2][L][L] quadrature matrices, transposed: MT[par][t'][t]
  float2* MT2 = nullptr;       // the same as float pairs (hi, lo)
  double* MR = nullptr;        // MW: [2][L][L] the same matrices row-major, MR[par][t][t'] (adjoints)
  float2* MR2 = nullptr;       // the same as float pairs
  double* wdiag = nullptr;     // DH: [nr] ring weights (null on MW)
  double2* tw = nullptr;       // [n] exp(+2 pi i e / n)
  float4* tw4 = nullptr;       // [n] the same as float pairs (re_hi, re_lo, im_hi, im_lo)
};

// Packed Wigner-d tables of one transform for the tensor-core contractions (kernels_tc.cu):
// fp16 or bf16 hi/lo pairs in 128-row x 64-deep core-matrix chunks.  Tile (m, n) starts at
// l0a = max(|m|,|n|) rounded down to 8.
struct TcTable {
  int Lb = 0;                  // beta rows of the inverse tables (rings rounded up to 128)
  int Lk = 0;                  // beta' reduction extent of the forward tables (rings rounded up to 64)
  int klf_max = 0;             // largest forward row extent
  int64_t* off_i = nullptr;    // device [Mc * nact] element offset of inverse tile (m, n)
  int64_t* off_f = nullptr;    // forward tile offsets
  int* kli = nullptr;          // device [Mc * nact] inverse l extent (multiple of 64; 0 if empty)
  int* klf = nullptr;          // forward l row extent (multiple of 128; 0 if empty)
  uint16_t *inv_hi = nullptr, *inv_lo = nullptr, *fwd_hi = nullptr, *fwd_lo = nullptr;
  int64_t op_i = 0, op_f = 0;  // prepared-operand elements per 16-map chunk (inverse, forward)
};

// Precomputed Wigner-d tables of one transform for the float64-accurate table contractions
// (kernels_tab.cu), float pairs.  Tile (m, n) covers l = l0a .. l0a + kp - 1 with
// l0a = max(|m|,|n|) rounded down to a multiple of 8 and kp a multiple of 32.
struct TabTable {
  int Lp = 0;                  // beta rows of the inverse tiles (rings rounded up to 64)
  int Lk = 0;                  // beta' rows of the forward tiles (rings rounded up to 32)
  int kpmax = 0;               // largest kp
  int64_t* off_inv = nullptr;  // device [Mc * nact] float2 offset of inverse tile (m, n): [kp][Lp]
  int64_t* off_fwd = nullptr;  // device [Mc * nact] offset of forward tile (m, n): [Lk][kp]
  int* kp = nullptr;           // device [Mc * nact] padded l extent (0 if l0 >= L)
  float2* inv = nullptr;       // d^l_mn(beta)
  float2* fwd = nullptr;       // (M^{par(m+n)})^T d^l_mn (MW) or w d^l_mn (DH), the quadrature folded in
  int64_t elems = 0;           // float2 elements of each of inv and fwd
};

// Sliced Wigner-d tables of one transform for the float64-accurate tensor-core contractions
// (kernels_tcx.cu, S2W_FP64_TC): seven bf16 slices per entry, in 128-row x 16-deep chunks with the
// slices of a chunk contiguous.
struct TcxTable {
  int Lb = 0;                  // beta rows of the inverse tables (rings rounded up to 128)
  int Lk = 0;                  // beta' reduction extent of the forward tables (rings rounded up to 16)
  int klf_max = 0;             // largest forward row extent
  int kli_max = 0;             // largest inverse K extent
  int lmin = 0;                // first l with a nonzero multiplier: tile (m, n) covers
                               // l >= max(|m|, |n|, lmin), starting at that rounded down to 8
  int64_t* off_i = nullptr;    // device [Mc * nact] element offset of inverse tile (m, n)
  int64_t* off_f = nullptr;    // forward tile offsets
  int64_t* opoff_i = nullptr;  // device [Mc * nact] offset of the inverse data slices of (m, n)
  int* kli = nullptr;          // device [Mc * nact] inverse l extent (multiple of 16; 0 if empty)
  int* klf = nullptr;          // forward l row extent (multiple of 128; 0 if empty)
  int* rexp_i = nullptr;       // device [Mc * nact][Lb] row exponents of the inverse tables
  int* rexp_f = nullptr;       // device [Mc * nact][klf_max] row exponents of the forward tables
  uint16_t *inv = nullptr, *fwd = nullptr;
  int64_t op_i = 0, op_f = 0;  // data-slice elements per 16-map chunk (inverse, forward)
};

// Sliced twiddle tables of the tensor-core DFTs (S2W_FP64_TC, kernels_dftx.cu) for one length
// n = 2L - 1 and one normalisation s: rows k = 0..L-1 (frequencies), reduction index p = 0..L-1
// (the index pairs p, n - p of the symmetric odd-length DFT), entries s cos(2 pi p k/n) and
// s sin(2 pi p k/n) as seven bf16 slices in 128-row x 16-deep chunks (the TcxTable layout).
struct DftxTable {
  int L = 0;
  int Kp = 0;                  // reduction extent: L rounded up to 16
  int Mt = 0;                  // row tiles of 128
  double scale = 1.0;
  int e = 0;                   // every entry |v| < 2^e
  uint16_t* cos = nullptr;
  uint16_t* sin = nullptr;
};

// Sliced n2-point table of the prime-factor tensor-core DFTs (S2W_FP64_TC, kernels_dftp.cu) for
// n = 2L - 1 = n1 n2 and one normalisation s: rows 2j / 2j + 1 = s cos / s sin(2 pi p2 j/n2),
// j <= (n2-1)/2, reduction index p2 < n2 (K rounded up to 16), seven bf16 slices in
// [chunk][slice][Rs x 16] core-matrix tiles; e1, e2 the output (CRT) index map.
struct DftpTable {
  int n = 0, n1 = 1, n2 = 1;
  int Rs = 0;                  // stored rows: n2 + 1 rounded up to 8
  int nkc = 0;                 // K chunks of 16
  int e = 0;                   // every entry |v| < 2^e
  int e1 = 0, e2 = 0;          // k = (k1 e1 + k2 e2) mod n
  double scale = 1.0;
  uint16_t* tab = nullptr;
};

// One Wigner / SHT transform instance: band-limit, the n values it carries and the
// per-(l, n) multipliers that fuse the harmonic products into the contraction.
struct TransformSpec {
  int L = 0, N = 0;          // band-limits (N = 1 for the SHT)
  int grid = -1;             // index into Plan::grids
  int nact = 0;              // number of n values carried
  int* nvals = nullptr;      // device [nact]
  std::vector<int> nvals_h;
  int lmin_h = 0;               // first l at which mult_inv or mult_fwd is nonzero for some n
  double2* mult_inv = nullptr;  // [L][nact] multiplier applied before the inverse contraction
  double2* mult_fwd = nullptr;  // [L][nact] multiplier applied after the forward contraction
  // mult_inv = minv_phase * minv_r with one complex phase for the whole transform (the
  // wavelet multipliers carry the constant factor xi of Eq. A8); minv_factored says it holds
  double* minv_r = nullptr;     // [L][nact] real factor
  double2 minv_phase{1.0, 0.0};
  bool minv_factored = false;
  double2* gphase = nullptr;    // [nact][2N-1] exp(+i n gamma_g)
  float4* gphase4 = nullptr;    // the same as float pairs
  double gscale = 1.0;          // gamma quadrature factor 2 pi/(2N-1) (1 for the SHT)
  // adjoint multipliers: the transposed products with the DFT normalisation moved across
  double2* adj_fwd = nullptr;   // [L][nact] conj(mult_inv) / ((2 pi/(2L-1)) gscale)
  double2* adj_inv = nullptr;   // [L][nact] conj(mult_fwd) * (2 pi/(2L-1)) gscale
  const TcTable* tc = nullptr;  // reduced-precision modes: packed tiles (shared between specs)
  const TabTable* tab = nullptr;  // precompute = 1: float64-accurate tables (shared between specs)
  const TcxTable* tcx = nullptr;  // S2W_FP64_TC: sliced tables (shared between specs)
  // S2W_FP64_TC: sliced twiddles of the tensor-core azimuthal DFTs (forward: normalisation
  // (2 pi/(2L-1)) gscale folded in; inverse: 1), null where the compensated DFTs run
  const DftxTable* dftx_fwd = nullptr;
  const DftxTable* dftx_inv = nullptr;
  // S2W_FP64_TC: the prime-factor tensor-core DFT tables (null where the length or the jobs do not
  // fit kernels_dftp.cu); where present this is the default form
  const DftpTable* dftp_fwd = nullptr;
  const DftpTable* dftp_inv = nullptr;
  // launch shapes chosen by s2w_plan_autotune (defaults otherwise)
  int dft_threads_fwd = 256, dft_threads_inv = 256;   // threads per block of the DFT kernels
  // S2W_FP64_TC: the form of the azimuthal DFTs, forward and inverse: kDftAuto (the prime-factor
  // tensor-core kernel where its tables exist, else the direct tensor-core GEMM where its tables
  // exist, else compensated float32), or one form forced by the autotuner
  int dft_form_fwd = 0, dft_form_inv = 0;
  int inv_mb = 16;                                     // maps per block of the inverse contraction
};

// A real Pout x Pin radial map of the ball sliced for the tensor cores (kernels_radx.cu): seven
// bf16 digits per entry, one exponent per row, [row tile][K chunk][slice][128 x 16].
struct RadxMap {
  int Pout = 0, Pin = 0, Mt = 0, nkc = 0;
  uint16_t* tab = nullptr;
  int* rexp = nullptr;
  int* kexp = nullptr;   // [Pin] power-of-two balancing exponents of the reduction index
};
void build_radx(const std::vector<double>& M, int Pout, int Pin, RadxMap* map, std::vector<uint16_t>& tab,
                std::vector<int>& rexp, std::vector<int>& kexp);
// data-slice workspace (uint16 elements) of a radial map over B maps of ncol complex columns
int64_t radx_ops_elems(int B, int Pin, int64_t ncol);
// out[b][o][c] (+)= wo[o][l] sum_q R[o][q] wi[q][l] in[b][q][c] (c = l Mc + m) on the tensor cores,
// float64-accurate; ops / fexp: workspaces of radx_ops_elems and B * L * Mc * 2 ints.
cudaError_t launch_radx(const RadxMap& R, const double2* in, double2* out, int B, int L, int Mc, const double* wi,
                        const double* wo, bool accumulate, uint16_t* ops, int* fexp, int* err, cudaStream_t st);

// DFT forms of S2W_FP64_TC (TransformSpec::dft_form_*; reported by s2w_plan_dft_forms)
enum DftForm { kDftAuto = 0, kDftComp = 1, kDftGemm = 2, kDftPfa = 3 };

struct s2w_plan_impl;

}  // namespace s2w

struct s2w_plan {
  s2w_params p{};
  bool native64 = false;               // every step in native float64 (S2W_FP64_NATIVE)
  int Mc = 0, mlo = 0;                 // m storage at L
  bool real = false;
  int nscales = 0, J = 0, L_phi = 1;
  int nr = 0;                          // colatitude rings at L (rings_of(p.sampling, L))
  std::vector<int> scale_j, Lj, Nj;
  std::vector<int64_t> wav_off;        // per map, elements
  int64_t map_elems = 0, wav_elems = 0, scal_elems = 0;

  std::vector<s2w::GridTables> grids;  // one per distinct band-limit
  s2w::TransformSpec sht;              // spin SHT at L (n = -spin)
  s2w::TransformSpec scal_t;           // scaling function synthesis at L_phi (n = 0)
  std::vector<s2w::TransformSpec> wav_t;   // wavelet scales (active n only, Psi multipliers)
  std::vector<s2w::TransformSpec> raw_t;   // raw Wigner transforms per scale (all n)

  bool tensor = false;                 // reduced-precision modes (S2W_FP32_SPLIT, S2W_BF16)
  std::vector<s2w::TcTable*> tc_tables;  // owned
  uint16_t *tc_b_hi = nullptr, *tc_b_lo = nullptr;   // prepared tensor-core operands (hi, lo)
  float* tc_scale = nullptr;                         // their power-of-two scales
  bool tcx = false;                    // float64-accurate tensor-core contractions (S2W_FP64_TC)
  std::vector<s2w::TcxTable*> tcx_tables;  // owned
  uint16_t* tcx_ops = nullptr;         // data slices of the current contraction
  int* tcx_fexp = nullptr;             // their column exponents
  std::vector<s2w::DftxTable*> dftx_tables;  // owned
  std::vector<s2w::DftpTable*> dftp_tables;  // owned
  uint16_t* dftx_ops = nullptr;        // data slices of the current tensor-core DFT
  int* dftx_fexp = nullptr;            // their column exponents
  uint16_t* dftp_ops = nullptr;        // prime-factor DFTs: data slices in pass order
  int* dftp_fexp = nullptr;            // their ring exponents
  float4* dftp_z = nullptr;            // inverse: Z staging between the GEMM and the gamma synthesis
  int cur_batch = 0;                   // > 0: maps per launch for an internal caller (ball transforms)
  bool precompute = false;             // float64-accurate table contractions (S2W_FP64, precompute = 1)
  std::vector<s2w::TabTable*> tab_tables;  // owned
  double2* flm_ws = nullptr;           // [batch][L][Mc] harmonic workspace
  double2* g_ws = nullptr;             // largest [batch][nact or 2N-1][rings_j][Mc_j] column buffer
  int64_t g_ws_elems = 0;
  int* err_word = nullptr;             // device error word
  int inject_timeout = 0;              // test hook: tensor-core contraction waits run out (s2w_plan_inject_timeout)
  // S2W_FP64_TC: the sliced GEMMs also sum the digit-pair diagonal 7 (34 digit pairs per K step
  // instead of 28, ~2^-47 instead of ~2^-44 of a term): the contractions and the direct-form DFTs; such
  // plans do not use the prime-factor DFT kernel (diagonals 0..6 only).  Set for the sphere plans
  // inside the ball plans, whose radial maps amplify the sphere transforms' error about a
  // hundredfold.
  int slice_diag7 = 0;
  cudaStream_t last_stream = nullptr;
  std::vector<void*> owned;            // every device allocation, freed on destroy
  std::vector<size_t> owned_bytes;     // their sizes
  int64_t workspace_bytes = 0;         // the part of them that is per-call scratch

  // tracing
  bool trace_on = false;
  std::vector<cudaEvent_t> trace_ev;   // pool, two per recorded launch
  struct TraceRec { int kind; double flops; };
  std::vector<TraceRec> trace_rec;
};

namespace s2w {

// Records a failure message for s2w_last_error() and returns s (api.cpp).
s2w_status record_error(s2w_status s, const std::string& msg);

// One transform's steps (api.cpp) with `batch` maps per launch: fwd = pixels -> harmonic
// accumulation (DFT, quadrature, contraction, products), inv = harmonic -> pixels, and their
// adjoints; coefficient strides come from the CoefArgs, pixel strides from pix_sb.
struct CoefArgs;
s2w_status run_fwd_transform(s2w_plan* P, const TransformSpec& t, const void* pix, int64_t pix_sb, CoefArgs out,
                             int batch, cudaStream_t st);
s2w_status run_inv_transform(s2w_plan* P, const TransformSpec& t, CoefArgs in, void* pix, int64_t pix_sb,
                             int batch, cudaStream_t st);
s2w_status run_adj_fwd_transform(s2w_plan* P, const TransformSpec& t, CoefArgs in, void* pix, int64_t pix_sb,
                                 int batch, cudaStream_t st);
s2w_status run_adj_inv_transform(s2w_plan* P, const TransformSpec& t, const void* pix, int64_t pix_sb,
                                 CoefArgs out, int batch, cudaStream_t st);

// Host-side plan construction (plan.cpp).
s2w_status build_plan(const s2w_params& p, cudaStream_t stream, s2w_plan* plan, std::string& err);
void free_plan(s2w_plan* plan);

// Kernel launchers (kernels_fp64.cu).  All asynchronous on `st`.
struct ColumnArgs {
  // A column buffer G[b][nact][nr][Mc] (complex) on the SO(3)/S2 grid at L with nr rings.
  double2* G;
  int B, nact, L, nr, Mc, mlo;
  // columns the float64 contractions launch (0: all Mc).  With G advanced by c0 columns and mlo
  // by c0, they cover the sub-range [c0, c0 + ncol) of a row of Mc (Mc stays the row stride).
  int ncol = 0;
};

// Pixel -> columns: azimuthal DFT (length 2L-1) and gamma DFT (length 2N-1), scaled by
// (2pi/(2L-1)) (2pi/(2N-1)).  Pixel layout [b][2N-1][nr][2L-1]; for the SHT N = 1.
// pix_sb = elements between consecutive maps of the pixel array.
cudaError_t launch_dft_forward(const s2w_plan* P, const GridTables& g, const TransformSpec& t,
                               const void* pix, int64_t pix_sb, bool real, ColumnArgs c, cudaStream_t st);
// Columns -> pixels: inverse gamma and alpha DFTs (no scaling).
cudaError_t launch_dft_inverse(const s2w_plan* P, const GridTables& g, const TransformSpec& t,
                               ColumnArgs c, void* pix, int64_t pix_sb, bool real, cudaStream_t st);

// Coefficient source for the inverse contraction: element (b, n_idx, l, m) is
// coef[b*s_b + n_idx*s_n + l*s_l + (m - mlo)] (s_n = 0 to share one f_lm across n).
struct CoefArgs {
  const double2* coef;   // written through (const_cast) when used as an output
  int64_t s_b, s_n, s_l;
  int mlo;
};
// G[b][n][beta][m] = sum_l coef(b,n,l,m) * mult_inv[l][n] * d^l_{m n}(beta)
cudaError_t launch_wigner_inverse(const s2w_plan* P, const GridTables& g, const TransformSpec& t,
                                  CoefArgs in, ColumnArgs out, cudaStream_t st);
// out(b,n,l,m) += mult_fwd[l][n] * sum_beta (M G)[beta] d^l_{m n}(beta), M the grid's colatitude
// quadrature (quad = false: the quadrature is skipped, G enters the sum as it is).
cudaError_t launch_wigner_forward(const s2w_plan* P, const GridTables& g, const TransformSpec& t,
                                  ColumnArgs in, CoefArgs out, cudaStream_t st, bool quad = true);
// In place on every column of c: G[b][n][.][m] <- M^T G[b][n][.][m], the transposed colatitude
// quadrature (adjoint of the forward transforms).
cudaError_t launch_quad_adjoint(const s2w_plan* P, const GridTables& g, const TransformSpec& t, ColumnArgs c,
                                cudaStream_t st);

cudaError_t launch_zero(void* p, int64_t bytes, cudaStream_t st);

// Tensor-core reduced-precision path (kernels_tc.cu).
struct TabTable;
cudaError_t launch_tc_pack(const TransformSpec& t, const TcTable& tab, const TabTable& src, int nr, int Mc, int mlo,
                           bool fp16, cudaStream_t st);
cudaError_t launch_tc_inverse(const s2w_plan* P, const GridTables& g, const TransformSpec& t, CoefArgs in,
                              ColumnArgs out, cudaStream_t st);
cudaError_t launch_tc_forward(const s2w_plan* P, const GridTables& g, const TransformSpec& t, ColumnArgs in,
                              CoefArgs out, cudaStream_t st);

// Float64-accurate tensor-core contractions by exact slicing (kernels_tcx.cu): table packing from
// float-pair tables, and the two contractions (same contracts as launch_wigner_inverse/forward).
struct TcxTable;
cudaError_t launch_tcx_pack(const TransformSpec& t, const TcxTable& tab, const TabTable& src, int nr, int Mc, int mlo,
                            cudaStream_t st);
cudaError_t launch_tcx_inverse(const s2w_plan* P, const GridTables& g, const TransformSpec& t, CoefArgs in,
                               ColumnArgs out, cudaStream_t st);
cudaError_t launch_tcx_forward(const s2w_plan* P, const GridTables& g, const TransformSpec& t, ColumnArgs in,
                               CoefArgs out, cudaStream_t st);

// Float64-accurate table contractions (kernels_tab.cu): build (recursion + folded quadrature)
// and the two contractions; same contracts as launch_wigner_inverse / launch_wigner_forward.
cudaError_t launch_tab_build(const GridTables& g, const TransformSpec& t, const TabTable& tab, int Mc, int mlo,
                             cudaStream_t st);
cudaError_t launch_tab_inverse(const GridTables& g, const TransformSpec& t, CoefArgs in, ColumnArgs out,
                               cudaStream_t st);
cudaError_t launch_tab_forward(const GridTables& g, const TransformSpec& t, ColumnArgs in, CoefArgs out,
                               cudaStream_t st);

// Tensor-core azimuthal DFTs of S2W_FP64_TC (kernels_dftx.cu); same contracts as
// launch_dft_forward / launch_dft_inverse.  dftx_shape_ok: the transform's carried n values fit
// (at most 16 jobs, the -n partner of every n for real maps, L <= 512, shared memory of the
// prologue kernels); the workspace sizes are for B maps on nr rings.
struct DftxTable;
bool dftx_shape_ok(const TransformSpec& t, bool real);
int64_t dftx_ops_elems(const TransformSpec& t, bool real, int B, int nr);
int64_t dftx_fexp_elems(int B, int nr);
void build_dftx_table(int L, double scale, DftxTable* tab, std::vector<uint16_t>& hcos, std::vector<uint16_t>& hsin);
cudaError_t launch_dftx_forward(const s2w_plan* P, const GridTables& g, const TransformSpec& t, const void* pix,
                                int64_t pix_sb, bool real, ColumnArgs c, cudaStream_t st);
cudaError_t launch_dftx_inverse(const s2w_plan* P, const GridTables& g, const TransformSpec& t, ColumnArgs c,
                                void* pix, int64_t pix_sb, bool real, cudaStream_t st);

// Prime-factor tensor-core azimuthal DFTs of S2W_FP64_TC (kernels_dftp.cu), same contracts as
// launch_dft_forward / launch_dft_inverse; no workspace.  dftp_shape: the factorisation n1 x n2 of
// 2L - 1 the kernel uses for this transform, false where none fits.
struct DftpTable;
bool dftp_shape(const TransformSpec& t, bool real, int* n1, int* n2);
void dftp_ws_elems(const TransformSpec& t, bool real, int n1, int B, int nr, int64_t* ops, int64_t* fexp, int64_t* z);
void build_dftp_table(int L, int n1, int n2, double scale, DftpTable* tab, std::vector<uint16_t>& h);
cudaError_t launch_dftp_forward(const s2w_plan* P, const GridTables& g, const TransformSpec& t, const void* pix,
                                int64_t pix_sb, bool real, ColumnArgs c, cudaStream_t st);
cudaError_t launch_dftp_inverse(const s2w_plan* P, const GridTables& g, const TransformSpec& t, ColumnArgs c,
                                void* pix, int64_t pix_sb, bool real, cudaStream_t st);
// The form a transform's DFTs run in (kDftComp, kDftGemm or kDftPfa) in S2W_FP64_TC.
int dft_form_used(const s2w_plan* P, const TransformSpec& t, bool fwd);

// The azimuthal DFTs of a transform in the plan's precision mode (api.cpp): plain float64,
// tensor-core (S2W_FP64_TC where the shape fits), or compensated / plain float32.
cudaError_t launch_dft_forward_mode(const s2w_plan* P, const GridTables& g, const TransformSpec& t, const void* pix,
                                    int64_t pix_sb, ColumnArgs c, cudaStream_t st);
cudaError_t launch_dft_inverse_mode(const s2w_plan* P, const GridTables& g, const TransformSpec& t, ColumnArgs c,
                                    void* pix, int64_t pix_sb, cudaStream_t st);

// Compensated-float32 versions of the two DFT launchers (kernels_dft_c32.cu); same contract.
// plain = ordinary float32 arithmetic (the reduced-precision modes).
cudaError_t launch_dftc_forward(const GridTables& g, const TransformSpec& t, const void* pix, int64_t pix_sb,
                                bool real, ColumnArgs c, cudaStream_t st, bool plain = false);
cudaError_t launch_dftc_inverse(const GridTables& g, const TransformSpec& t, ColumnArgs c, void* pix,
                                int64_t pix_sb, bool real, cudaStream_t st, bool plain = false);
// The plain-float32 DFTs of the reduced-precision modes (kernels_dftf.cu): usable when the
// shape fits their shared-memory layout; launch_dftc_* take them for plain = true.
bool dftf_usable(const GridTables& g, const TransformSpec& t, bool real, bool fwd);
cudaError_t launch_dftf_forward(const GridTables& g, const TransformSpec& t, const void* pix, int64_t pix_sb,
                                bool real, ColumnArgs c, cudaStream_t st);
cudaError_t launch_dftf_inverse(const GridTables& g, const TransformSpec& t, ColumnArgs c, void* pix,
                                int64_t pix_sb, bool real, cudaStream_t st);

}  // namespace s2w
