// Directional scale-discretised wavelet transform on the ball (Sec. 3.2; operators of Sec. 5.1
// and Algorithm 2; dictionary App. A.3-A.4; radial multiresolution Sec. 3.3).
//
// Psi^{jj'}_lnp = Psi^j_ln kappa^{j'}(p) factors into the sphere wavelet and a radial tiling, so
// every step maps onto the sphere plan's transforms run over a batch of radial nodes plus
// small radial maps (kernels_radial.cu):
//   analysis   F(r_i)  = Y f(r_i)                      spin-0 SHT of every node map
//              f_p     = sum_i omega_i K_p(r_i) F(r_i)  Laguerre transform (Z = K Y)
//              W^Phi   = Y^-1 sum_p K_p(r_i) phi_lp f_p  phi_lp = sqrt(4 pi/(2l+1)) Phi_l0p
//              g^{j'}(r'_i) = sum_p K_p(r'_i) kappa^{j'}(p) f_p   on the P_j'-node rule r'
//              W^{jj'}(r'_i) = sphere inverse Wigner of scale j applied to g^{j'}(r'_i)
//   synthesis  the transposed sequence with the forward transforms, then Z^-1.
// The scaling function is read as |Phi_l0p|^2 (4 pi/(2l+1)) = A + B - A B with
// A = k_lambda(l/lambda^J0), B = k_nu(p/nu^J0'), which satisfies the admissibility condition of
// Sec. 3.2 exactly (the printed hybrid generator does not).
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "s2w_internal.h"
#include "tiling.h"

namespace s2w {
cudaError_t launch_radial_gen(const float2* R2, const double2* in, double2* out, int B, int Pout, int Pin, int L,
                              int Mc, const double* wi, const double* wo, bool accumulate, cudaStream_t st);
void laguerre_rule(int P, double tau, int kmax, std::vector<double>& r, std::vector<double>& omega,
                   std::vector<double>& K);
}  // namespace s2w

struct s2w_ball_wav_plan {
  s2w_ball_wav_params p{};
  s2w_plan* sph = nullptr;            // sphere wavelet plan over batch * P node maps
  int Mc = 0, Jr = 0;
  std::vector<int> jr, Pj;            // radial scales j' and their rules P_j'
  std::vector<int> sc_s, sc_r;        // wavelet scale k = (sphere scale index, radial index)
  std::vector<int64_t> wav_off;       // element offsets of the scale blocks (whole batch)
  int64_t field_elems = 0, wav_elems = 0;
  float2 *Rf = nullptr, *Ri = nullptr, *RfT = nullptr, *RiT = nullptr;   // full rule, P x P
  std::vector<float2*> Ra, Rs, RaT, RsT;   // per radial scale: [Pj][P], [P][Pj] and transposes
  // tensor-core precision modes (S2W_FP32_SPLIT, S2W_BF16, S2W_FP64_TC): the same maps sliced for
  // the tensor cores (kernels_radx.cu), index-aligned with the pairs above, and their workspaces
  bool tc = false;
  s2w::RadxMap RfX, RiX, RfTX, RiTX;
  std::vector<s2w::RadxMap> RaX, RsX, RaTX, RsTX;
  uint16_t* rops = nullptr;
  int* rfexp = nullptr;
  double* phi = nullptr;              // [P][L]
  double2* fhat = nullptr;            // [batch][P][L][Mc]
  double2* ws = nullptr;              // [batch * P][L][Mc]
  std::vector<void*> owned;
};

namespace {

using namespace s2w;

template <class T>
s2w_status upload_vec(s2w_ball_wav_plan* W, const std::vector<T>& h, T** d, cudaStream_t st) {
  void* q = nullptr;
  if (cudaMalloc(&q, std::max<size_t>(h.size(), 1) * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return record_error(S2W_ENOMEM, "cudaMalloc failed for a ball wavelet table");
  }
  W->owned.push_back(q);
  if (!h.empty() && cudaMemcpyAsync(q, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return record_error(S2W_ECUDA, "upload of a ball wavelet table failed");
  *d = static_cast<T*>(q);
  return S2W_OK;
}

// rows x cols float64 matrix -> float pairs, and its transpose
void pairs(const std::vector<double>& M, int rows, int cols, std::vector<float2>& out, std::vector<float2>& outT) {
  out.resize((size_t)rows * cols);
  outT.resize((size_t)rows * cols);
  for (int i = 0; i < rows; ++i)
    for (int k = 0; k < cols; ++k) {
      const double v = M[(size_t)i * cols + k];
      const float h = (float)v;
      const float2 pr = make_float2(h, (float)(v - (double)h));
      out[(size_t)i * cols + k] = pr;
      outT[(size_t)k * rows + i] = pr;
    }
}

void destroy(s2w_ball_wav_plan* W) {
  if (W->sph) s2w_plan_destroy(W->sph);
  for (void* q : W->owned) cudaFree(q);
  delete W;
}

s2w_status check_ptr(const void* q, const char* name) {
  if (q == nullptr) return record_error(S2W_EINVAL, std::string(name) + " is NULL");
  if (reinterpret_cast<uintptr_t>(q) % 8 != 0) return record_error(S2W_EINVAL, std::string(name) + " is misaligned");
  return S2W_OK;
}

#define BW_CUDA(call, what)                                                                 \
  do {                                                                                      \
    cudaError_t _e = (call);                                                                \
    if (_e != cudaSuccess) return record_error(S2W_ECUDA, std::string(what) + ": " + cudaGetErrorString(_e)); \
  } while (0)
#define BW_TRY(x)                  \
  do {                             \
    s2w_status _s = (x);           \
    if (_s != S2W_OK) return _s;   \
  } while (0)

struct Ctx {
  s2w_ball_wav_plan* W;
  cudaStream_t st;
  int B, P, L, Mc;
  int64_t ncol() const { return (int64_t)L * Mc; }
  size_t elem() const { return W->p.reality ? sizeof(double) : sizeof(double2); }
  CoefArgs coef(double2* c) const {
    CoefArgs a;
    a.coef = c;
    a.s_b = ncol();
    a.s_n = 0;
    a.s_l = Mc;
    a.mlo = W->sph->mlo;
    return a;
  }
  s2w_status zero(double2* q, int64_t rows) const {
    BW_CUDA(cudaMemsetAsync(q, 0, (size_t)rows * ncol() * sizeof(double2), st), "zero workspace");
    return S2W_OK;
  }
  // one radial map: on the tensor cores (RX, float64-accurate) in the tensor-core precision modes,
  // else the compensated SIMT kernel on the float pairs R
  s2w_status radial(const float2* R, const s2w::RadxMap& RX, const double2* in, double2* out, int Pout, int Pin,
                    const double* wi, const double* wo, bool acc) const {
    if (W->tc)
      BW_CUDA(launch_radx(RX, in, out, B, L, Mc, wi, wo, acc, W->rops, W->rfexp, W->sph->err_word, st), "radial map");
    else
      BW_CUDA(launch_radial_gen(R, in, out, B, Pout, Pin, L, Mc, wi, wo, acc, st), "radial map");
    return S2W_OK;
  }
  int64_t scale_pix(int k) const {   // elements of one node map of wavelet scale k
    const int s = W->sc_s[k];
    const int Lj = W->sph->Lj[s], Nj = W->sph->Nj[s];
    return (int64_t)(2 * Nj - 1) * rings_of(W->p.sampling, Lj) * (2 * Lj - 1);
  }
  char* wav_at(void* wav, int k) const { return static_cast<char*>(wav) + W->wav_off[k] * elem(); }
};

}  // namespace

extern "C" {

s2w_status s2w_ball_wav_plan_create(const s2w_ball_wav_params* prm, void* stream, s2w_ball_wav_plan** out) {
  if (out == nullptr) return record_error(S2W_EINVAL, "out is NULL");
  *out = nullptr;
  if (prm == nullptr) return record_error(S2W_EINVAL, "params is NULL");
  const s2w_ball_wav_params p = *prm;
  if (p.P < 2 || p.P > 256) return record_error(S2W_EINVAL, "P must satisfy 2 <= P <= 256");
  if (!(p.nu > 1.0) || !std::isfinite(p.nu)) return record_error(S2W_EINVAL, "nu must be > 1");
  if (!(p.tau > 0.0) || !std::isfinite(p.tau)) return record_error(S2W_EINVAL, "tau must be > 0");
  if (p.batch < 1) return record_error(S2W_EINVAL, "batch must be >= 1");
  if (p.spin != 0) return record_error(S2W_EUNSUPPORTED, "the ball wavelet transform supports spin 0");
  int Jr = 0;
  while (tiling::ceil_pow(p.nu, Jr) < p.P) ++Jr;
  if (p.J0r < 0 || p.J0r > Jr) return record_error(S2W_EINVAL, "J0r must satisfy 0 <= J0r <= J'");
  s2w_ball_wav_plan* W = new (std::nothrow) s2w_ball_wav_plan();
  if (W == nullptr) return record_error(S2W_ENOMEM, "host allocation failed");
  W->p = p;
  W->Jr = Jr;
  s2w_params sp{};
  sp.L = p.L;
  sp.N = p.N;
  sp.J0 = p.J0;
  sp.spin = 0;
  sp.reality = p.reality;
  sp.batch = p.batch * p.P;
  sp.precision = p.precision;
  sp.precompute = p.precompute;
  sp.lambda = p.lambda;
  sp.sampling = p.sampling;
  s2w_status s = s2w_plan_create(&sp, stream, &W->sph);   // validates L, N, lambda, J0
  if (s != S2W_OK) {
    delete W;
    return s;
  }
  // the radial maps amplify the sphere transforms' error about a hundredfold: in S2W_FP64_TC the
  // sliced GEMMs of this plan also sum the digit-pair diagonal 7
  W->sph->slice_diag7 = 1;
  cudaStream_t st = (cudaStream_t)stream;
  const int P = p.P, L = p.L;
  W->Mc = p.reality ? L : 2 * L - 1;
  W->field_elems = (int64_t)P * rings_of(p.sampling, L) * (2 * L - 1);
  for (int j = p.J0r; j <= Jr; ++j) {
    W->jr.push_back(j);
    W->Pj.push_back(std::min(tiling::ceil_pow(p.nu, j + 1), P));
  }
  W->wav_off.assign(1, 0);
  for (int s_ = 0; s_ < W->sph->nscales; ++s_)
    for (size_t r = 0; r < W->jr.size(); ++r) {
      W->sc_s.push_back(s_);
      W->sc_r.push_back((int)r);
      const int Lj = W->sph->Lj[s_], Nj = W->sph->Nj[s_];
      W->wav_off.push_back(W->wav_off.back() +
                           (int64_t)p.batch * W->Pj[r] * (2 * Nj - 1) * rings_of(p.sampling, Lj) * (2 * Lj - 1));
    }
  W->wav_elems = W->wav_off.back();

  // full rule and the per-scale radial maps, float64 on the host
  tiling::Tiling tl(p.lambda), tn(p.nu);
  std::vector<double> r, om, K;
  laguerre_rule(P, p.tau, P, r, om, K);
  std::vector<double> Rf((size_t)P * P), Ri((size_t)P * P), phi((size_t)P * L);
  for (int i = 0; i < P; ++i)
    for (int k = 0; k < P; ++k) {
      Rf[(size_t)k * P + i] = om[i] * K[(size_t)i * P + k];
      Ri[(size_t)i * P + k] = K[(size_t)i * P + k];
    }
  const double sl = std::pow(p.lambda, p.J0), sn = std::pow(p.nu, p.J0r);
  for (int q = 0; q < P; ++q) {
    const double Bq = tn.k(q / sn);
    for (int l = 0; l < L; ++l) {
      const double A = tl.k(l / sl);
      phi[(size_t)q * L + l] = std::sqrt(std::max(0.0, A + Bq - A * Bq));
    }
  }
  W->tc = p.precision == S2W_FP32_SPLIT || p.precision == S2W_BF16 || p.precision == S2W_FP64_TC;
  // a rows x cols map and its transpose, sliced for the tensor cores (tensor-core modes only)
  auto sliced = [&](const std::vector<double>& M, int rows, int cols, RadxMap* X, RadxMap* XT) -> s2w_status {
    if (!W->tc) return S2W_OK;
    std::vector<double> MT((size_t)rows * cols);
    for (int i = 0; i < rows; ++i)
      for (int k = 0; k < cols; ++k) MT[(size_t)k * rows + i] = M[(size_t)i * cols + k];
    std::vector<uint16_t> tab;
    std::vector<int> rexp, kexp;
    s2w_status s2;
    build_radx(M, rows, cols, X, tab, rexp, kexp);
    if ((s2 = upload_vec(W, tab, &X->tab, st)) || (s2 = upload_vec(W, rexp, &X->rexp, st)) ||
        (s2 = upload_vec(W, kexp, &X->kexp, st)))
      return s2;
    build_radx(MT, cols, rows, XT, tab, rexp, kexp);
    if ((s2 = upload_vec(W, tab, &XT->tab, st)) || (s2 = upload_vec(W, rexp, &XT->rexp, st)) ||
        (s2 = upload_vec(W, kexp, &XT->kexp, st)))
      return s2;
    return S2W_OK;
  };
  std::vector<float2> a2, a2T;
  if ((s = upload_vec(W, phi, &W->phi, st))) return destroy(W), s;
  pairs(Rf, P, P, a2, a2T);
  if ((s = upload_vec(W, a2, &W->Rf, st)) || (s = upload_vec(W, a2T, &W->RfT, st))) return destroy(W), s;
  if ((s = sliced(Rf, P, P, &W->RfX, &W->RfTX))) return destroy(W), s;
  pairs(Ri, P, P, a2, a2T);
  if ((s = upload_vec(W, a2, &W->Ri, st)) || (s = upload_vec(W, a2T, &W->RiT, st))) return destroy(W), s;
  if ((s = sliced(Ri, P, P, &W->RiX, &W->RiTX))) return destroy(W), s;
  W->Ra.resize(W->jr.size());
  W->RaT.resize(W->jr.size());
  W->Rs.resize(W->jr.size());
  W->RsT.resize(W->jr.size());
  W->RaX.resize(W->jr.size());
  W->RaTX.resize(W->jr.size());
  W->RsX.resize(W->jr.size());
  W->RsTX.resize(W->jr.size());
  for (size_t ri = 0; ri < W->jr.size(); ++ri) {
    const int Pr = W->Pj[ri];
    std::vector<double> rr, oo, KK;
    laguerre_rule(Pr, p.tau, Pr, rr, oo, KK);
    const double sc = std::pow(p.nu, W->jr[ri]);
    std::vector<double> Ra((size_t)Pr * P, 0.0), Rs((size_t)P * Pr, 0.0);
    for (int q = 0; q < Pr; ++q) {
      const double kap = tn.kappa(q / sc);   // zero for q >= nu^{j'+1}
      for (int i = 0; i < Pr; ++i) {
        Ra[(size_t)i * P + q] = KK[(size_t)i * Pr + q] * kap;
        Rs[(size_t)q * Pr + i] = kap * oo[i] * KK[(size_t)i * Pr + q];
      }
    }
    pairs(Ra, Pr, P, a2, a2T);
    if ((s = upload_vec(W, a2, &W->Ra[ri], st)) || (s = upload_vec(W, a2T, &W->RaT[ri], st))) return destroy(W), s;
    if ((s = sliced(Ra, Pr, P, &W->RaX[ri], &W->RaTX[ri]))) return destroy(W), s;
    pairs(Rs, P, Pr, a2, a2T);
    if ((s = upload_vec(W, a2, &W->Rs[ri], st)) || (s = upload_vec(W, a2T, &W->RsT[ri], st))) return destroy(W), s;
    if ((s = sliced(Rs, P, Pr, &W->RsX[ri], &W->RsTX[ri]))) return destroy(W), s;
  }
  if (W->tc) {   // data-slice workspace of the largest map (K = P input nodes), column exponents
    const int64_t ncol = (int64_t)L * W->Mc;
    std::vector<uint16_t> ops((size_t)radx_ops_elems(p.batch, P, ncol), 0);
    std::vector<int> fx((size_t)p.batch * ncol * 2, 0);
    if ((s = upload_vec(W, ops, &W->rops, st)) || (s = upload_vec(W, fx, &W->rfexp, st))) return destroy(W), s;
  }
  void* q = nullptr;
  const size_t cb = (size_t)p.batch * P * L * W->Mc * sizeof(double2);
  if (cudaMalloc(&q, cb) != cudaSuccess) return cudaGetLastError(), destroy(W), record_error(S2W_ENOMEM, "ball workspace");
  W->owned.push_back(q);
  W->fhat = static_cast<double2*>(q);
  if (cudaMalloc(&q, cb) != cudaSuccess) return cudaGetLastError(), destroy(W), record_error(S2W_ENOMEM, "ball workspace");
  W->owned.push_back(q);
  W->ws = static_cast<double2*>(q);
  if (cudaStreamSynchronize(st) != cudaSuccess) return destroy(W), record_error(S2W_ECUDA, "ball wavelet plan upload");
  *out = W;
  return S2W_OK;
}

s2w_status s2w_ball_wav_plan_destroy(s2w_ball_wav_plan* W) {
  if (W == nullptr) return record_error(S2W_EINVAL, "plan is NULL");
  destroy(W);
  return S2W_OK;
}

s2w_status s2w_ball_wav_query_layout(const s2w_ball_wav_plan* W, int64_t* field_elems, int64_t* wav_elems,
                                     int* nscales, int* j, int* jr, int64_t* wav_offsets, int* Lj, int* Nj,
                                     int* Pj) {
  if (W == nullptr) return record_error(S2W_EINVAL, "plan is NULL");
  const int n = (int)W->sc_s.size();
  if (field_elems) *field_elems = W->field_elems;
  if (wav_elems) *wav_elems = W->wav_elems;
  if (nscales) *nscales = n;
  for (int k = 0; k < n; ++k) {
    const int s = W->sc_s[k], r = W->sc_r[k];
    if (j) j[k] = W->sph->scale_j[s];
    if (jr) jr[k] = W->jr[r];
    if (wav_offsets) wav_offsets[k] = W->wav_off[k];
    if (Lj) Lj[k] = W->sph->Lj[s];
    if (Nj) Nj[k] = W->sph->Nj[s];
    if (Pj) Pj[k] = W->Pj[r];
  }
  if (wav_offsets) wav_offsets[n] = W->wav_off[n];
  return S2W_OK;
}

s2w_status s2w_ball_forward(const s2w_ball_wav_plan* cW, const void* f, void* wav, void* scal, void* stream) {
  if (cW == nullptr) return record_error(S2W_EINVAL, "plan is NULL");
  s2w_ball_wav_plan* W = const_cast<s2w_ball_wav_plan*>(cW);
  BW_TRY(check_ptr(f, "f"));
  BW_TRY(check_ptr(wav, "wav"));
  BW_TRY(check_ptr(scal, "scal"));
  Ctx c{W, (cudaStream_t)stream, W->p.batch, W->p.P, W->p.L, W->Mc};
  s2w_plan* S = W->sph;
  S->last_stream = c.st;
  const int nb = c.B * c.P;
  // f_p = K Y f
  BW_TRY(c.zero(W->ws, nb));
  BW_TRY(run_fwd_transform(S, S->sht, f, S->map_elems, c.coef(W->ws), nb, c.st));
  BW_TRY(c.radial(W->Rf, W->RfX, W->ws, W->fhat, c.P, c.P, nullptr, nullptr, false));
  // W^Phi = Y^-1 K^-1 (phi f_p)
  BW_TRY(c.radial(W->Ri, W->RiX, W->fhat, W->ws, c.P, c.P, W->phi, nullptr, false));
  BW_TRY(run_inv_transform(S, S->sht, c.coef(W->ws), scal, S->map_elems, nb, c.st));
  // W^{jj'} = D^-1_j (conj Psi^j  g^{j'}),  g^{j'} = K'^-1 (kappa^{j'} f_p)
  for (size_t r = 0; r < W->jr.size(); ++r) {
    const int Pr = W->Pj[r];
    BW_TRY(c.radial(W->Ra[r], W->RaX[r], W->fhat, W->ws, Pr, c.P, nullptr, nullptr, false));
    for (size_t k = 0; k < W->sc_s.size(); ++k) {
      if (W->sc_r[k] != (int)r) continue;
      BW_TRY(run_inv_transform(S, S->wav_t[W->sc_s[k]], c.coef(W->ws), c.wav_at(wav, (int)k), c.scale_pix((int)k),
                               c.B * Pr, c.st));
    }
  }
  return S2W_OK;
}

s2w_status s2w_ball_inverse(const s2w_ball_wav_plan* cW, const void* wav, const void* scal, void* f, void* stream) {
  if (cW == nullptr) return record_error(S2W_EINVAL, "plan is NULL");
  s2w_ball_wav_plan* W = const_cast<s2w_ball_wav_plan*>(cW);
  BW_TRY(check_ptr(f, "f"));
  BW_TRY(check_ptr(wav, "wav"));
  BW_TRY(check_ptr(scal, "scal"));
  Ctx c{W, (cudaStream_t)stream, W->p.batch, W->p.P, W->p.L, W->Mc};
  s2w_plan* S = W->sph;
  S->last_stream = c.st;
  const int nb = c.B * c.P;
  // f_p = phi K Y W^Phi
  BW_TRY(c.zero(W->ws, nb));
  BW_TRY(run_fwd_transform(S, S->sht, scal, S->map_elems, c.coef(W->ws), nb, c.st));
  BW_TRY(c.radial(W->Rf, W->RfX, W->ws, W->fhat, c.P, c.P, nullptr, W->phi, false));
  // f_p += kappa^{j'} K' sum_j (Psi^j D_j W^{jj'})
  for (size_t r = 0; r < W->jr.size(); ++r) {
    const int Pr = W->Pj[r];
    BW_TRY(c.zero(W->ws, c.B * Pr));
    for (size_t k = 0; k < W->sc_s.size(); ++k) {
      if (W->sc_r[k] != (int)r) continue;
      BW_TRY(run_fwd_transform(S, S->wav_t[W->sc_s[k]], c.wav_at(const_cast<void*>(wav), (int)k), c.scale_pix((int)k),
                               c.coef(W->ws), c.B * Pr, c.st));
    }
    BW_TRY(c.radial(W->Rs[r], W->RsX[r], W->ws, W->fhat, c.P, Pr, nullptr, nullptr, true));
  }
  // f = Y^-1 K^-1 f_p
  BW_TRY(c.radial(W->Ri, W->RiX, W->fhat, W->ws, c.P, c.P, nullptr, nullptr, false));
  return run_inv_transform(S, S->sht, c.coef(W->ws), f, S->map_elems, nb, c.st);
}

s2w_status s2w_ball_forward_adjoint(const s2w_ball_wav_plan* cW, const void* gwav, const void* gscal, void* gf,
                                    void* stream) {
  if (cW == nullptr) return record_error(S2W_EINVAL, "plan is NULL");
  s2w_ball_wav_plan* W = const_cast<s2w_ball_wav_plan*>(cW);
  BW_TRY(check_ptr(gf, "gf"));
  BW_TRY(check_ptr(gwav, "gwav"));
  BW_TRY(check_ptr(gscal, "gscal"));
  Ctx c{W, (cudaStream_t)stream, W->p.batch, W->p.P, W->p.L, W->Mc};
  s2w_plan* S = W->sph;
  S->last_stream = c.st;
  const int nb = c.B * c.P;
  // scaling branch: g_p = phi K^-T (Y^-1)^H gscal
  BW_TRY(c.zero(W->ws, nb));
  BW_TRY(run_adj_inv_transform(S, S->sht, gscal, S->map_elems, c.coef(W->ws), nb, c.st));
  BW_TRY(c.radial(W->RiT, W->RiTX, W->ws, W->fhat, c.P, c.P, nullptr, W->phi, false));
  // wavelet branch: g_p += (K'^-1 kappa)^T sum_j (D_j^-1 conj Psi^j)^H gwav^{jj'}
  for (size_t r = 0; r < W->jr.size(); ++r) {
    const int Pr = W->Pj[r];
    BW_TRY(c.zero(W->ws, c.B * Pr));
    for (size_t k = 0; k < W->sc_s.size(); ++k) {
      if (W->sc_r[k] != (int)r) continue;
      BW_TRY(run_adj_inv_transform(S, S->wav_t[W->sc_s[k]], c.wav_at(const_cast<void*>(gwav), (int)k),
                                   c.scale_pix((int)k), c.coef(W->ws), c.B * Pr, c.st));
    }
    BW_TRY(c.radial(W->RaT[r], W->RaTX[r], W->ws, W->fhat, c.P, Pr, nullptr, nullptr, true));
  }
  // gf = Y^H K^T g_p
  BW_TRY(c.radial(W->RfT, W->RfTX, W->fhat, W->ws, c.P, c.P, nullptr, nullptr, false));
  return run_adj_fwd_transform(S, S->sht, c.coef(W->ws), gf, S->map_elems, nb, c.st);
}

s2w_status s2w_ball_inverse_adjoint(const s2w_ball_wav_plan* cW, const void* gf, void* gwav, void* gscal,
                                    void* stream) {
  if (cW == nullptr) return record_error(S2W_EINVAL, "plan is NULL");
  s2w_ball_wav_plan* W = const_cast<s2w_ball_wav_plan*>(cW);
  BW_TRY(check_ptr(gf, "gf"));
  BW_TRY(check_ptr(gwav, "gwav"));
  BW_TRY(check_ptr(gscal, "gscal"));
  Ctx c{W, (cudaStream_t)stream, W->p.batch, W->p.P, W->p.L, W->Mc};
  s2w_plan* S = W->sph;
  S->last_stream = c.st;
  const int nb = c.B * c.P;
  // g_p = K^-T (Y^-1)^H gf
  BW_TRY(c.zero(W->ws, nb));
  BW_TRY(run_adj_inv_transform(S, S->sht, gf, S->map_elems, c.coef(W->ws), nb, c.st));
  BW_TRY(c.radial(W->RiT, W->RiTX, W->ws, W->fhat, c.P, c.P, nullptr, nullptr, false));
  // gscal = Y^H K^T (phi g_p)
  BW_TRY(c.radial(W->RfT, W->RfTX, W->fhat, W->ws, c.P, c.P, W->phi, nullptr, false));
  BW_TRY(run_adj_fwd_transform(S, S->sht, c.coef(W->ws), gscal, S->map_elems, nb, c.st));
  // gwav^{jj'} = (Psi^j D_j)^H (kappa K')^T g_p
  for (size_t r = 0; r < W->jr.size(); ++r) {
    const int Pr = W->Pj[r];
    BW_TRY(c.radial(W->RsT[r], W->RsTX[r], W->fhat, W->ws, Pr, c.P, nullptr, nullptr, false));
    for (size_t k = 0; k < W->sc_s.size(); ++k) {
      if (W->sc_r[k] != (int)r) continue;
      BW_TRY(run_adj_fwd_transform(S, S->wav_t[W->sc_s[k]], c.coef(W->ws), c.wav_at(gwav, (int)k),
                                   c.scale_pix((int)k), c.B * Pr, c.st));
    }
  }
  return S2W_OK;
}

s2w_status s2w_ball_wav_check(const s2w_ball_wav_plan* W) {
  if (W == nullptr) return record_error(S2W_EINVAL, "plan is NULL");
  return s2w_check(W->sph);
}

s2w_status s2w_ball_wav_plan_autotune(s2w_ball_wav_plan* W, void* stream) {
  if (W == nullptr) return record_error(S2W_EINVAL, "plan is NULL");
  return s2w_plan_autotune(W->sph, stream);
}

}  // extern "C"
