// C ABI (include/s2w.h): plan lifetime, layout queries and the execute calls that
// sequence the kernels of one transform on the caller's stream.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>

#include "s2w_internal.h"

using namespace s2w;

namespace {

thread_local std::string g_last_error;

s2w_status fail(s2w_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

s2w_status cuda_fail(cudaError_t e, const char* where) {
  return fail(S2W_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define S2W_CUDA(call, where)                          \
  do {                                                 \
    cudaError_t _e = (call);                           \
    if (_e != cudaSuccess) return cuda_fail(_e, where); \
  } while (0)

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

s2w_status check_ptr(const void* p, bool real_elems, const char* name) {
  if (p == nullptr) return fail(S2W_EINVAL, std::string(name) + " is NULL");
  if (!aligned(p, real_elems ? 8 : 16)) return fail(S2W_EINVAL, std::string(name) + " is misaligned");
  return S2W_OK;
}

int Mc_at(const s2w_plan* P, int L) { return P->real ? L : 2 * L - 1; }
// maps per launch: the plan's batch unless an internal caller (the ball transforms) runs a
// different number of maps through the plan's transforms
int batch_of(const s2w_plan* P) { return P->cur_batch > 0 ? P->cur_batch : P->p.batch; }
int mlo_at(const s2w_plan* P, int L) { return P->real ? 0 : -(L - 1); }

const GridTables& grid_of(const s2w_plan* P, const TransformSpec& t) { return P->grids[t.grid]; }

CoefArgs flm_ws_args(const s2w_plan* P) {
  CoefArgs c;
  c.coef = P->flm_ws;
  c.s_b = (int64_t)P->p.L * P->Mc;
  c.s_n = 0;
  c.s_l = P->Mc;
  c.mlo = P->mlo;
  return c;
}

ColumnArgs cols(const s2w_plan* P, int nact, int L) {
  ColumnArgs c;
  c.G = P->g_ws;
  c.B = batch_of(P);
  c.nact = nact;
  c.L = L;
  c.nr = rings_of(P->p.sampling, L);
  c.Mc = Mc_at(P, L);
  c.mlo = mlo_at(P, L);
  return c;
}

// ---- tracing: events around each launch plus its algorithmic float64 operation count
enum Kind { K_DFT_FWD = 0, K_DFT_INV = 1, K_WIG_INV = 2, K_WIG_FWD = 3, K_QUAD_ADJ = 4, K_NKINDS = 5 };
const char* kKindNames[K_NKINDS] = {"dft_forward", "dft_inverse", "wigner_inverse", "wigner_forward",
                                    "quadrature_adjoint"};

double contraction_terms(const s2w_plan* P, const TransformSpec& t) {
  const int L = t.L, mlo = mlo_at(P, L), Mc = Mc_at(P, L), nr = rings_of(P->p.sampling, L);
  double T = 0.0;
  for (int mi = 0; mi < Mc; ++mi)
    for (int n : t.nvals_h) {
      const int l0 = std::max(std::abs(mlo + mi), std::abs(n));
      if (l0 < L) T += double(nr) * double(L - l0);
    }
  return T;
}

double dft_flops(const s2w_plan* P, const TransformSpec& t) {
  const double n = 2.0 * t.L - 1.0, B = batch_of(P), Ng = 2.0 * t.N - 1.0, nr = rings_of(P->p.sampling, t.L);
  const double ring = (P->real ? 2.5 : 5.0) * n * std::log2(n);
  return B * Ng * nr * ring + 8.0 * B * nr * Mc_at(P, t.L) * t.nact * Ng;
}

// algorithmic flops per contraction term: the recursion step (5, unless the d values come
// from precomputed tables) plus a complex-times-real multiply-add (4) per map
double term_flops(const s2w_plan* P, const TransformSpec& t) {
  return (t.tab || t.tc || t.tcx ? 0.0 : 5.0) + 4.0 * batch_of(P);
}

struct TraceScope {
  s2w_plan* P;
  cudaStream_t st;
  bool on = false;
  size_t slot = 0;
  TraceScope(s2w_plan* P_, cudaStream_t st_, int kind, double flops) : P(P_), st(st_) {
    if (!P->trace_on) return;
    slot = 2 * P->trace_rec.size();
    if (slot + 2 > P->trace_ev.size()) return;
    on = true;
    cudaEventRecord(P->trace_ev[slot], st);
    P->trace_rec.push_back({kind, flops});
  }
  ~TraceScope() {
    if (on) cudaEventRecord(P->trace_ev[slot + 1], st);
  }
};

// pixels -> harmonic accumulation: out += mult_fwd * (forward transform of pix)
s2w_status fwd_transform(s2w_plan* P, const TransformSpec& t, const void* pix, int64_t pix_sb, CoefArgs out,
                         cudaStream_t st) {
  const GridTables& g = grid_of(P, t);
  ColumnArgs c = cols(P, t.nact, t.L);
  {
    TraceScope ts(P, st, K_DFT_FWD, P->trace_on ? dft_flops(P, t) : 0.0);
    S2W_CUDA(launch_dft_forward_mode(P, g, t, pix, pix_sb, c, st), "azimuthal DFT (forward)");
  }
  {
    TraceScope ts(P, st, K_WIG_FWD, P->trace_on ? contraction_terms(P, t) * term_flops(P, t) : 0.0);
    S2W_CUDA(t.tcx   ? launch_tcx_forward(P, g, t, c, out, st)
             : t.tc  ? launch_tc_forward(P, g, t, c, out, st)
             : t.tab ? launch_tab_forward(g, t, c, out, st)
                     : launch_wigner_forward(P, g, t, c, out, st),
             "forward contraction");
  }
  return S2W_OK;
}

// harmonic -> pixels: pix = inverse transform of (mult_inv * coef)
s2w_status inv_transform(s2w_plan* P, const TransformSpec& t, CoefArgs in, void* pix, int64_t pix_sb,
                         cudaStream_t st) {
  const GridTables& g = grid_of(P, t);
  ColumnArgs c = cols(P, t.nact, t.L);
  {
    TraceScope ts(P, st, K_WIG_INV, P->trace_on ? contraction_terms(P, t) * term_flops(P, t) : 0.0);
    S2W_CUDA(t.tcx   ? launch_tcx_inverse(P, g, t, in, c, st)
             : t.tc  ? launch_tc_inverse(P, g, t, in, c, st)
             : (t.tab && t.minv_factored) ? launch_tab_inverse(g, t, in, c, st)
                     : launch_wigner_inverse(P, g, t, in, c, st),
             "inverse contraction");
  }
  {
    TraceScope ts(P, st, K_DFT_INV, P->trace_on ? dft_flops(P, t) : 0.0);
    S2W_CUDA(launch_dft_inverse_mode(P, g, t, c, pix, pix_sb, st), "azimuthal DFT (inverse)");
  }
  return S2W_OK;
}

// ---- adjoints: each step of fwd_transform / inv_transform transposed, in reverse order.
// The contractions run on the float64-accurate kernels in every mode (tc = nullptr); the
// products are conjugated and carry the DFT normalisation moved across (adj_fwd, adj_inv).

// Adjoint of inv_transform: out += adj_fwd * (contraction over beta, no quadrature) of the
// forward DFT of pix.
s2w_status adj_inv_transform(s2w_plan* P, const TransformSpec& t, const void* pix, int64_t pix_sb, CoefArgs out,
                             cudaStream_t st) {
  const GridTables& g = grid_of(P, t);
  ColumnArgs c = cols(P, t.nact, t.L);
  TransformSpec ta = t;
  ta.mult_fwd = t.adj_fwd;
  ta.tc = nullptr;
  ta.tab = nullptr;
  ta.tcx = nullptr;
  {
    TraceScope ts(P, st, K_DFT_FWD, P->trace_on ? dft_flops(P, t) : 0.0);
    S2W_CUDA(P->native64 ? launch_dft_forward(P, g, ta, pix, pix_sb, P->real, c, st)
                         : launch_dftc_forward(g, ta, pix, pix_sb, P->real, c, st, false),
             "azimuthal DFT (adjoint of the inverse DFT)");
  }
  {
    TraceScope ts(P, st, K_WIG_FWD, P->trace_on ? contraction_terms(P, t) * (5.0 + 4.0 * batch_of(P)) : 0.0);
    S2W_CUDA(launch_wigner_forward(P, g, ta, c, out, st, false), "adjoint of the inverse contraction");
  }
  return S2W_OK;
}

// Adjoint of fwd_transform: pix = inverse DFT of the transposed quadrature of the inverse
// contraction of (adj_inv * coef).
s2w_status adj_fwd_transform(s2w_plan* P, const TransformSpec& t, CoefArgs in, void* pix, int64_t pix_sb,
                             cudaStream_t st) {
  const GridTables& g = grid_of(P, t);
  ColumnArgs c = cols(P, t.nact, t.L);
  TransformSpec ta = t;
  ta.mult_inv = t.adj_inv;
  ta.tc = nullptr;
  ta.tab = nullptr;
  ta.tcx = nullptr;
  {
    TraceScope ts(P, st, K_WIG_INV, P->trace_on ? contraction_terms(P, t) * (5.0 + 4.0 * batch_of(P)) : 0.0);
    S2W_CUDA(launch_wigner_inverse(P, g, ta, in, c, st), "adjoint of the forward contraction");
  }
  {
    const double nr = rings_of(P->p.sampling, t.L);
    TraceScope ts(P, st, K_QUAD_ADJ,
                  P->trace_on ? (g.wdiag ? 2.0 : 4.0 * t.L) * batch_of(P) * t.nact * (double)Mc_at(P, t.L) * nr : 0.0);
    S2W_CUDA(launch_quad_adjoint(P, g, ta, c, st), "transposed colatitude quadrature");
  }
  {
    TraceScope ts(P, st, K_DFT_INV, P->trace_on ? dft_flops(P, t) : 0.0);
    S2W_CUDA(P->native64 ? launch_dft_inverse(P, g, ta, c, pix, pix_sb, P->real, st)
                         : launch_dftc_inverse(g, ta, c, pix, pix_sb, P->real, st, false),
             "azimuthal DFT (adjoint of the forward DFT)");
  }
  return S2W_OK;
}

size_t pix_bytes(const s2w_plan* P) { return P->real ? sizeof(double) : sizeof(double2); }

}  // namespace

namespace s2w {
int dft_form_used(const s2w_plan* P, const TransformSpec& t, bool fwd) {
  if (!P->tcx && t.tcx == nullptr) return kDftComp;   // the reduced modes' wavelet scales
  const int f = fwd ? t.dft_form_fwd : t.dft_form_inv;
  // the prime-factor kernel sums the digit-pair diagonals 0..6 only: plans that also sum
  // diagonal 7 (the ball's) take the direct form
  const bool pfa = !P->slice_diag7 && (fwd ? (const void*)t.dftp_fwd : (const void*)t.dftp_inv) != nullptr;
  const bool gemm = (fwd ? (const void*)t.dftx_fwd : (const void*)t.dftx_inv) != nullptr;
  if (f == kDftComp) return kDftComp;
  if (f == kDftPfa && pfa) return kDftPfa;
  if (f == kDftGemm && gemm) return kDftGemm;
  return pfa ? kDftPfa : gemm ? kDftGemm : kDftComp;
}

cudaError_t launch_dft_forward_mode(const s2w_plan* P, const GridTables& g, const TransformSpec& t, const void* pix,
                                    int64_t pix_sb, ColumnArgs c, cudaStream_t st) {
  if (P->native64) return launch_dft_forward(P, g, t, pix, pix_sb, P->real, c, st);
  switch (dft_form_used(P, t, true)) {
    case kDftPfa: return launch_dftp_forward(P, g, t, pix, pix_sb, P->real, c, st);
    case kDftGemm: return launch_dftx_forward(P, g, t, pix, pix_sb, P->real, c, st);
    default: return launch_dftc_forward(g, t, pix, pix_sb, P->real, c, st, t.tc != nullptr);
  }
}

cudaError_t launch_dft_inverse_mode(const s2w_plan* P, const GridTables& g, const TransformSpec& t, ColumnArgs c,
                                    void* pix, int64_t pix_sb, cudaStream_t st) {
  if (P->native64) return launch_dft_inverse(P, g, t, c, pix, pix_sb, P->real, st);
  switch (dft_form_used(P, t, false)) {
    case kDftPfa: return launch_dftp_inverse(P, g, t, c, pix, pix_sb, P->real, st);
    case kDftGemm: return launch_dftx_inverse(P, g, t, c, pix, pix_sb, P->real, st);
    default: return launch_dftc_inverse(g, t, c, pix, pix_sb, P->real, st, t.tc != nullptr);
  }
}

// Lets other translation units report through s2w_last_error().
s2w_status record_error(s2w_status s, const std::string& msg) { return fail(s, msg); }

// The per-transform steps for other translation units, with `batch` maps per launch.
struct BatchScope {
  s2w_plan* P;
  BatchScope(s2w_plan* P_, int b) : P(P_) { P->cur_batch = b; }
  ~BatchScope() { P->cur_batch = 0; }
};
s2w_status run_fwd_transform(s2w_plan* P, const TransformSpec& t, const void* pix, int64_t pix_sb, CoefArgs out,
                             int batch, cudaStream_t st) {
  BatchScope bs(P, batch);
  return fwd_transform(P, t, pix, pix_sb, out, st);
}
s2w_status run_inv_transform(s2w_plan* P, const TransformSpec& t, CoefArgs in, void* pix, int64_t pix_sb,
                             int batch, cudaStream_t st) {
  BatchScope bs(P, batch);
  return inv_transform(P, t, in, pix, pix_sb, st);
}
s2w_status run_adj_fwd_transform(s2w_plan* P, const TransformSpec& t, CoefArgs in, void* pix, int64_t pix_sb,
                                 int batch, cudaStream_t st) {
  BatchScope bs(P, batch);
  return adj_fwd_transform(P, t, in, pix, pix_sb, st);
}
s2w_status run_adj_inv_transform(s2w_plan* P, const TransformSpec& t, const void* pix, int64_t pix_sb,
                                 CoefArgs out, int batch, cudaStream_t st) {
  BatchScope bs(P, batch);
  return adj_inv_transform(P, t, pix, pix_sb, out, st);
}
}  // namespace s2w

extern "C" {

const char* s2w_last_error(void) { return g_last_error.c_str(); }

const char* s2w_version(void) { return "s2w-gb300 0.1 (sm_103a, float64)"; }

s2w_status s2w_plan_device_bytes(const s2w_plan* P, int64_t* table_bytes, int64_t* workspace_bytes) {
  if (P == nullptr) return s2w::record_error(S2W_EINVAL, "plan is NULL");
  int64_t tot = 0;
  for (size_t b : P->owned_bytes) tot += (int64_t)b;
  if (table_bytes) *table_bytes = tot - P->workspace_bytes;
  if (workspace_bytes) *workspace_bytes = P->workspace_bytes;
  return S2W_OK;
}

s2w_status s2w_plan_create(const s2w_params* params, void* stream, s2w_plan** out) {
  if (out == nullptr) return fail(S2W_EINVAL, "out is NULL");
  *out = nullptr;
  if (params == nullptr) return fail(S2W_EINVAL, "params is NULL");
  s2w_plan* P = new (std::nothrow) s2w_plan();
  if (P == nullptr) return fail(S2W_ENOMEM, "host allocation failed");
  std::string err;
  s2w_status s = build_plan(*params, (cudaStream_t)stream, P, err);
  if (s != S2W_OK) {
    free_plan(P);
    delete P;
    return fail(s, err);
  }
  P->last_stream = (cudaStream_t)stream;
  *out = P;
  g_last_error.clear();
  return S2W_OK;
}

s2w_status s2w_plan_destroy(s2w_plan* plan) {
  if (plan == nullptr) return fail(S2W_EINVAL, "plan is NULL");
  for (cudaEvent_t e : plan->trace_ev) cudaEventDestroy(e);
  plan->trace_ev.clear();
  free_plan(plan);
  delete plan;
  return S2W_OK;
}

s2w_status s2w_query_layout(const s2w_plan* P, int64_t* map_elems, int64_t* wav_elems, int64_t* scal_elems,
                            int* nscales, int64_t* wav_offsets, int* Lj, int* Nj, int* L_phi) {
  if (P == nullptr) return fail(S2W_EINVAL, "plan is NULL");
  if (map_elems) *map_elems = P->map_elems;
  if (wav_elems) *wav_elems = P->wav_elems;
  if (scal_elems) *scal_elems = P->scal_elems;
  if (nscales) *nscales = P->nscales;
  if (L_phi) *L_phi = P->L_phi;
  for (int s = 0; s < P->nscales; ++s) {
    if (wav_offsets) wav_offsets[s] = P->wav_off[s];
    if (Lj) Lj[s] = P->Lj[s];
    if (Nj) Nj[s] = P->Nj[s];
  }
  if (wav_offsets) wav_offsets[P->nscales] = P->wav_off[P->nscales];
  return S2W_OK;
}

s2w_status s2w_forward(const s2w_plan* cP, const void* f, void* wav, void* scal, void* stream) {
  if (cP == nullptr) return fail(S2W_EINVAL, "plan is NULL");
  s2w_plan* P = const_cast<s2w_plan*>(cP);
  s2w_status s;
  if ((s = check_ptr(f, P->real, "f")) || (s = check_ptr(wav, P->real, "wav")) ||
      (s = check_ptr(scal, P->real, "scal")))
    return s;
  cudaStream_t st = (cudaStream_t)stream;
  P->last_stream = st;
  const int64_t B = P->p.batch;
  // f_lm = Y f  (Eq. 2)
  S2W_CUDA(launch_zero(P->flm_ws, B * (int64_t)P->p.L * P->Mc * sizeof(double2), st), "zero f_lm");
  if ((s = fwd_transform(P, P->sht, f, P->map_elems, flm_ws_args(P), st))) return s;
  // scaling map W^Phi = Y^-1 (Phi f_lm) at L_Phi  (Eq. 41)
  if ((s = inv_transform(P, P->scal_t, flm_ws_args(P), scal, P->scal_elems, st))) return s;
  // wavelet maps W^j = D^-1 (N Psi^j f_lm) at (L_j, N_j)  (Eq. 40)
  char* wbase = static_cast<char*>(wav);
  for (int sc = 0; sc < P->nscales; ++sc) {
    void* pix = wbase + P->wav_off[sc] * pix_bytes(P);
    if ((s = inv_transform(P, P->wav_t[sc], flm_ws_args(P), pix, P->wav_elems, st))) return s;
  }
  return S2W_OK;
}

s2w_status s2w_inverse(const s2w_plan* cP, const void* wav, const void* scal, void* f, void* stream) {
  if (cP == nullptr) return fail(S2W_EINVAL, "plan is NULL");
  s2w_plan* P = const_cast<s2w_plan*>(cP);
  s2w_status s;
  if ((s = check_ptr(f, P->real, "f")) || (s = check_ptr(wav, P->real, "wav")) ||
      (s = check_ptr(scal, P->real, "scal")))
    return s;
  cudaStream_t st = (cudaStream_t)stream;
  P->last_stream = st;
  const int64_t B = P->p.batch;
  S2W_CUDA(launch_zero(P->flm_ws, B * (int64_t)P->p.L * P->Mc * sizeof(double2), st), "zero f_lm");
  // f_lm = Phi Y W^Phi + sum_j Psi^j+ D W^j  (Eq. 42)
  if ((s = fwd_transform(P, P->scal_t, scal, P->scal_elems, flm_ws_args(P), st))) return s;
  const char* wbase = static_cast<const char*>(wav);
  for (int sc = 0; sc < P->nscales; ++sc) {
    const void* pix = wbase + P->wav_off[sc] * pix_bytes(P);
    if ((s = fwd_transform(P, P->wav_t[sc], pix, P->wav_elems, flm_ws_args(P), st))) return s;
  }
  // f = Y^-1 f_lm
  return inv_transform(P, P->sht, flm_ws_args(P), f, P->map_elems, st);
}

s2w_status s2w_forward_adjoint(const s2w_plan* cP, const void* gwav, const void* gscal, void* gf, void* stream) {
  if (cP == nullptr) return fail(S2W_EINVAL, "plan is NULL");
  s2w_plan* P = const_cast<s2w_plan*>(cP);
  s2w_status s;
  if ((s = check_ptr(gf, P->real, "gf")) || (s = check_ptr(gwav, P->real, "gwav")) ||
      (s = check_ptr(gscal, P->real, "gscal")))
    return s;
  cudaStream_t st = (cudaStream_t)stream;
  P->last_stream = st;
  const int64_t B = P->p.batch;
  S2W_CUDA(launch_zero(P->flm_ws, B * (int64_t)P->p.L * P->Mc * sizeof(double2), st), "zero f_lm");
  // g_lm = sum over the scaling map and the scales of (Y^-1 Phi)^H gscal, (D^-1 N Psi^j)^H gwav^j
  if ((s = adj_inv_transform(P, P->scal_t, gscal, P->scal_elems, flm_ws_args(P), st))) return s;
  const char* wbase = static_cast<const char*>(gwav);
  for (int sc = 0; sc < P->nscales; ++sc) {
    const void* pix = wbase + P->wav_off[sc] * pix_bytes(P);
    if ((s = adj_inv_transform(P, P->wav_t[sc], pix, P->wav_elems, flm_ws_args(P), st))) return s;
  }
  // gf = Y^H g_lm
  return adj_fwd_transform(P, P->sht, flm_ws_args(P), gf, P->map_elems, st);
}

s2w_status s2w_inverse_adjoint(const s2w_plan* cP, const void* gf, void* gwav, void* gscal, void* stream) {
  if (cP == nullptr) return fail(S2W_EINVAL, "plan is NULL");
  s2w_plan* P = const_cast<s2w_plan*>(cP);
  s2w_status s;
  if ((s = check_ptr(gf, P->real, "gf")) || (s = check_ptr(gwav, P->real, "gwav")) ||
      (s = check_ptr(gscal, P->real, "gscal")))
    return s;
  cudaStream_t st = (cudaStream_t)stream;
  P->last_stream = st;
  const int64_t B = P->p.batch;
  // g_lm = (Y^-1)^H gf
  S2W_CUDA(launch_zero(P->flm_ws, B * (int64_t)P->p.L * P->Mc * sizeof(double2), st), "zero f_lm");
  if ((s = adj_inv_transform(P, P->sht, gf, P->map_elems, flm_ws_args(P), st))) return s;
  // gscal = (Phi Y)^H g_lm, gwav^j = (Psi^j+ D)^H g_lm
  if ((s = adj_fwd_transform(P, P->scal_t, flm_ws_args(P), gscal, P->scal_elems, st))) return s;
  char* wbase = static_cast<char*>(gwav);
  for (int sc = 0; sc < P->nscales; ++sc) {
    void* pix = wbase + P->wav_off[sc] * pix_bytes(P);
    if ((s = adj_fwd_transform(P, P->wav_t[sc], flm_ws_args(P), pix, P->wav_elems, st))) return s;
  }
  return S2W_OK;
}

s2w_status s2w_sht_forward(const s2w_plan* cP, const void* f, void* flm, void* stream) {
  if (cP == nullptr) return fail(S2W_EINVAL, "plan is NULL");
  s2w_plan* P = const_cast<s2w_plan*>(cP);
  s2w_status s;
  if ((s = check_ptr(f, P->real, "f")) || (s = check_ptr(flm, false, "flm"))) return s;
  cudaStream_t st = (cudaStream_t)stream;
  P->last_stream = st;
  CoefArgs out = flm_ws_args(P);
  out.coef = static_cast<double2*>(flm);
  S2W_CUDA(launch_zero(flm, (int64_t)P->p.batch * P->p.L * P->Mc * sizeof(double2), st), "zero flm");
  return fwd_transform(P, P->sht, f, P->map_elems, out, st);
}

s2w_status s2w_sht_inverse(const s2w_plan* cP, const void* flm, void* f, void* stream) {
  if (cP == nullptr) return fail(S2W_EINVAL, "plan is NULL");
  s2w_plan* P = const_cast<s2w_plan*>(cP);
  s2w_status s;
  if ((s = check_ptr(f, P->real, "f")) || (s = check_ptr(flm, false, "flm"))) return s;
  cudaStream_t st = (cudaStream_t)stream;
  P->last_stream = st;
  CoefArgs in = flm_ws_args(P);
  in.coef = static_cast<const double2*>(flm);
  return inv_transform(P, P->sht, in, f, P->map_elems, st);
}

// ---- m-sharded spin SHT: the stages of s2w_sht_inverse / s2w_sht_forward on a range of m
// columns or of rings, on the float64-accurate on-the-fly kernels of every mode.

s2w_status s2w_shard_layout(int L, int spin, int reality, int sampling, int nranks, int rank, int* c_begin,
                            int* c_end, int* ring_begin, int* ring_end) {
  if (L < 2 || nranks < 1 || rank < 0 || rank >= nranks) return fail(S2W_EINVAL, "need L >= 2 and 0 <= rank < nranks");
  if (std::abs(spin) >= L || (reality && spin != 0)) return fail(S2W_EINVAL, "need |spin| < L (0 for real maps)");
  if (sampling != S2W_SAMPLING_MW && sampling != S2W_SAMPLING_DH) return fail(S2W_EINVAL, "unknown sampling");
  const int Mc = reality ? L : 2 * L - 1, mlo = reality ? 0 : -(L - 1), as = std::abs(spin);
  // contraction work of column c: the degrees l = max(|m|, |spin|) .. L-1 (at least one)
  auto cost = [&](int c) { return (int64_t)(L - std::max(std::abs(mlo + c), as)); };
  int64_t total = 0;
  for (int c = 0; c < Mc; ++c) total += cost(c);
  // first column of part r: the smallest c whose preceding work reaches r/nranks of the total
  auto bound = [&](int r) {
    if (r >= nranks) return Mc;
    int64_t cum = 0;
    for (int c = 0; c < Mc; ++c) {
      if (cum * nranks >= (int64_t)r * total) return c;
      cum += cost(c);
    }
    return Mc;
  };
  const int nr = rings_of(sampling, L);
  if (c_begin) *c_begin = bound(rank);
  if (c_end) *c_end = bound(rank + 1);
  if (ring_begin) *ring_begin = (int)((int64_t)rank * nr / nranks);
  if (ring_end) *ring_end = (int)((int64_t)(rank + 1) * nr / nranks);
  return S2W_OK;
}

}  // extern "C"

namespace {

// the SHT's transform with every tensor-core and table path switched off: the recursion kernels
TransformSpec shard_spec(const s2w_plan* P) {
  TransformSpec t = P->sht;
  t.tc = nullptr;
  t.tab = nullptr;
  t.tcx = nullptr;
  return t;
}

s2w_status shard_args(const s2w_plan* P, const void* a, bool a_real, const char* an, const void* b, bool b_real,
                      const char* bn, int begin, int end, int limit) {
  if (P == nullptr) return fail(S2W_EINVAL, "plan is NULL");
  s2w_status s;
  if ((s = check_ptr(a, a_real, an)) || (s = check_ptr(b, b_real, bn))) return s;
  if (begin < 0 || begin > end || end > limit) return fail(S2W_EINVAL, "range outside 0 <= begin <= end <= limit");
  return S2W_OK;
}

// column args for columns [c0, c1) of a [batch][R(L)][Mc] buffer
ColumnArgs shard_cols(const s2w_plan* P, const TransformSpec& t, void* G, int c0, int c1) {
  ColumnArgs c = cols(P, t.nact, P->p.L);
  c.B = P->p.batch;
  c.G = static_cast<double2*>(G) + c0;
  c.mlo += c0;
  c.ncol = c1 - c0;
  return c;
}

// one map's rows [r0, r1) of a [batch][R(L)][Mc] buffer, and the matching pixel rings
ColumnArgs shard_rows(const s2w_plan* P, const TransformSpec& t, const void* G, int b, int r0, int r1) {
  ColumnArgs c = cols(P, t.nact, P->p.L);
  c.B = 1;
  c.G = const_cast<double2*>(static_cast<const double2*>(G)) + ((int64_t)b * c.nr + r0) * c.Mc;
  c.nr = r1 - r0;
  return c;
}
char* shard_pix(const s2w_plan* P, const void* f, int b, int r0) {
  const size_t el = P->real ? sizeof(double) : sizeof(double2);
  return const_cast<char*>(static_cast<const char*>(f)) +
         ((int64_t)b * P->map_elems + (int64_t)r0 * (2 * P->p.L - 1)) * el;
}

}  // namespace

extern "C" {

s2w_status s2w_sht_inverse_columns(const s2w_plan* cP, const void* flm, void* cols_, int c_begin, int c_end,
                                   void* stream) {
  s2w_status s;
  if ((s = shard_args(cP, flm, false, "flm", cols_, false, "cols", c_begin, c_end, cP ? cP->Mc : 0))) return s;
  if (c_begin == c_end) return S2W_OK;
  s2w_plan* P = const_cast<s2w_plan*>(cP);
  cudaStream_t st = (cudaStream_t)stream;
  P->last_stream = st;
  const TransformSpec t = shard_spec(P);
  CoefArgs in = flm_ws_args(P);
  in.coef = static_cast<const double2*>(flm);
  S2W_CUDA(launch_wigner_inverse(P, grid_of(P, t), t, in, shard_cols(P, t, cols_, c_begin, c_end), st),
           "inverse contraction (column range)");
  return S2W_OK;
}

s2w_status s2w_sht_inverse_rings(const s2w_plan* cP, const void* cols_, void* f, int ring_begin, int ring_end,
                                 void* stream) {
  s2w_status s;
  const int nr = cP ? rings_of(cP->p.sampling, cP->p.L) : 0;
  if ((s = shard_args(cP, cols_, false, "cols", f, cP && cP->real, "f", ring_begin, ring_end, nr))) return s;
  if (ring_begin == ring_end) return S2W_OK;
  s2w_plan* P = const_cast<s2w_plan*>(cP);
  cudaStream_t st = (cudaStream_t)stream;
  P->last_stream = st;
  const TransformSpec t = shard_spec(P);
  const GridTables& g = grid_of(P, t);
  for (int b = 0; b < P->p.batch; ++b) {
    const ColumnArgs c = shard_rows(P, t, cols_, b, ring_begin, ring_end);
    void* pix = shard_pix(P, f, b, ring_begin);
    S2W_CUDA(P->native64 ? launch_dft_inverse(P, g, t, c, pix, P->map_elems, P->real, st)
                         : launch_dftc_inverse(g, t, c, pix, P->map_elems, P->real, st, false),
             "azimuthal DFT (inverse, ring range)");
  }
  return S2W_OK;
}

s2w_status s2w_sht_forward_rings(const s2w_plan* cP, const void* f, void* cols_, int ring_begin, int ring_end,
                                 void* stream) {
  s2w_status s;
  const int nr = cP ? rings_of(cP->p.sampling, cP->p.L) : 0;
  if ((s = shard_args(cP, f, cP && cP->real, "f", cols_, false, "cols", ring_begin, ring_end, nr))) return s;
  if (ring_begin == ring_end) return S2W_OK;
  s2w_plan* P = const_cast<s2w_plan*>(cP);
  cudaStream_t st = (cudaStream_t)stream;
  P->last_stream = st;
  const TransformSpec t = shard_spec(P);
  const GridTables& g = grid_of(P, t);
  for (int b = 0; b < P->p.batch; ++b) {
    const ColumnArgs c = shard_rows(P, t, cols_, b, ring_begin, ring_end);
    const void* pix = shard_pix(P, f, b, ring_begin);
    S2W_CUDA(P->native64 ? launch_dft_forward(P, g, t, pix, P->map_elems, P->real, c, st)
                         : launch_dftc_forward(g, t, pix, P->map_elems, P->real, c, st, false),
             "azimuthal DFT (forward, ring range)");
  }
  return S2W_OK;
}

s2w_status s2w_sht_forward_columns(const s2w_plan* cP, const void* cols_, void* flm, int c_begin, int c_end,
                                   void* stream) {
  s2w_status s;
  if ((s = shard_args(cP, cols_, false, "cols", flm, false, "flm", c_begin, c_end, cP ? cP->Mc : 0))) return s;
  if (c_begin == c_end) return S2W_OK;
  s2w_plan* P = const_cast<s2w_plan*>(cP);
  cudaStream_t st = (cudaStream_t)stream;
  P->last_stream = st;
  const TransformSpec t = shard_spec(P);
  // the contraction accumulates: clear this range's coefficients of every (map, l) first
  S2W_CUDA(cudaMemset2DAsync(static_cast<double2*>(flm) + c_begin, (size_t)P->Mc * sizeof(double2), 0,
                             (size_t)(c_end - c_begin) * sizeof(double2), (size_t)P->p.batch * P->p.L, st),
           "zero flm (column range)");
  CoefArgs out = flm_ws_args(P);
  out.coef = static_cast<double2*>(flm);
  S2W_CUDA(launch_wigner_forward(P, grid_of(P, t), t,
                                 shard_cols(P, t, const_cast<void*>(cols_), c_begin, c_end), out, st),
           "forward contraction (column range)");
  return S2W_OK;
}

static CoefArgs raw_args(const s2w_plan* P, int sc, const void* flmn) {
  const int Lj = P->Lj[sc], Nj = P->Nj[sc], Mcj = Mc_at(P, Lj);
  CoefArgs c;
  c.coef = static_cast<const double2*>(flmn);
  c.s_l = Mcj;
  c.s_n = (int64_t)Lj * Mcj;
  c.s_b = (int64_t)(2 * Nj - 1) * Lj * Mcj;
  c.mlo = mlo_at(P, Lj);
  return c;
}

s2w_status s2w_wigner_forward(const s2w_plan* cP, int scale, const void* f, void* flmn, void* stream) {
  if (cP == nullptr) return fail(S2W_EINVAL, "plan is NULL");
  s2w_plan* P = const_cast<s2w_plan*>(cP);
  if (scale < 0 || scale >= P->nscales) return fail(S2W_EINVAL, "scale index out of range");
  if (P->tensor) return fail(S2W_EUNSUPPORTED, "the raw Wigner transforms run in the float64 modes only");
  s2w_status s;
  if ((s = check_ptr(f, P->real, "f")) || (s = check_ptr(flmn, false, "flmn"))) return s;
  cudaStream_t st = (cudaStream_t)stream;
  P->last_stream = st;
  CoefArgs out = raw_args(P, scale, flmn);
  S2W_CUDA(launch_zero(flmn, out.s_b * P->p.batch * (int64_t)sizeof(double2), st), "zero flmn");
  const int Lj = P->Lj[scale], Nj = P->Nj[scale];
  return fwd_transform(P, P->raw_t[scale], f, (int64_t)(2 * Nj - 1) * rings_of(P->p.sampling, Lj) * (2 * Lj - 1),
                       out, st);
}

s2w_status s2w_wigner_inverse(const s2w_plan* cP, int scale, const void* flmn, void* f, void* stream) {
  if (cP == nullptr) return fail(S2W_EINVAL, "plan is NULL");
  s2w_plan* P = const_cast<s2w_plan*>(cP);
  if (scale < 0 || scale >= P->nscales) return fail(S2W_EINVAL, "scale index out of range");
  if (P->tensor) return fail(S2W_EUNSUPPORTED, "the raw Wigner transforms run in the float64 modes only");
  s2w_status s;
  if ((s = check_ptr(f, P->real, "f")) || (s = check_ptr(flmn, false, "flmn"))) return s;
  cudaStream_t st = (cudaStream_t)stream;
  P->last_stream = st;
  const int Lj = P->Lj[scale], Nj = P->Nj[scale];
  return inv_transform(P, P->raw_t[scale], raw_args(P, scale, flmn), f,
                       (int64_t)(2 * Nj - 1) * rings_of(P->p.sampling, Lj) * (2 * Lj - 1), st);
}

s2w_status s2w_check(const s2w_plan* P) {
  if (P == nullptr) return fail(S2W_EINVAL, "plan is NULL");
  cudaError_t e = cudaStreamSynchronize(P->last_stream);
  if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
  int word = 0;
  e = cudaMemcpy(&word, P->err_word, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "error word read");
  if (word != 0) {
    cudaMemset(P->err_word, 0, sizeof(int));
    return fail((s2w_status)word, "device error word set");
  }
  return S2W_OK;
}

s2w_status s2w_plan_inject_timeout(s2w_plan* P, int on) {
  if (P == nullptr) return fail(S2W_EINVAL, "plan is NULL");
  P->inject_timeout = on ? 1 : 0;
  return S2W_OK;
}

s2w_status s2w_trace_enable(s2w_plan* P, int on, int capacity) {
  if (P == nullptr) return fail(S2W_EINVAL, "plan is NULL");
  if (on && capacity < 1) return fail(S2W_EINVAL, "capacity must be >= 1");
  P->trace_on = false;
  if (on) {
    const size_t want = 2 * (size_t)capacity;
    while (P->trace_ev.size() < want) {
      cudaEvent_t e;
      cudaError_t err = cudaEventCreate(&e);
      if (err != cudaSuccess) return cuda_fail(err, "cudaEventCreate");
      P->trace_ev.push_back(e);
    }
    P->trace_rec.clear();
    P->trace_rec.reserve(capacity);
    P->trace_on = true;
  }
  return S2W_OK;
}

s2w_status s2w_trace_reset(s2w_plan* P) {
  if (P == nullptr) return fail(S2W_EINVAL, "plan is NULL");
  P->trace_rec.clear();
  return S2W_OK;
}

s2w_status s2w_trace_read(const s2w_plan* P, int kind, int64_t* launches, double* ms, double* flops) {
  if (P == nullptr) return fail(S2W_EINVAL, "plan is NULL");
  if (kind < 0 || kind >= K_NKINDS) return fail(S2W_EINVAL, "kernel kind out of range");
  int64_t n = 0;
  double t = 0.0, f = 0.0;
  for (size_t i = 0; i < P->trace_rec.size(); ++i) {
    if (P->trace_rec[i].kind != kind) continue;
    cudaError_t e = cudaEventSynchronize(P->trace_ev[2 * i + 1]);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
    float dt = 0.0f;
    e = cudaEventElapsedTime(&dt, P->trace_ev[2 * i], P->trace_ev[2 * i + 1]);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime");
    ++n;
    t += dt;
    f += P->trace_rec[i].flops;
  }
  if (launches) *launches = n;
  if (ms) *ms = t;
  if (flops) *flops = f;
  return S2W_OK;
}

const char* s2w_kernel_name(int kind) { return (kind >= 0 && kind < K_NKINDS) ? kKindNames[kind] : ""; }

}  // extern "C"
