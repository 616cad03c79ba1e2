// Ball transforms: the Fourier-Laguerre radial transform (Sec. 2.3, Eqs. 6-8) and the
// spherical-Laguerre transform Z = K o Y (Eqs. 9-11) on generalised Gauss-Laguerre nodes.
//
// Radial quadrature (host, float64): the nodes x_i are the P roots of L^(2)_P, found by
// Sturm-sequence bisection on the Jacobi matrix of the weight x^2 e^-x and polished with
// Newton steps on the three-term Laguerre recurrence; r_i = tau x_i.  With Gamma(P+3)/P! =
// (P+1)(P+2), the Gauss weights are w_i = (P+2) x_i / ((P+1) L^(2)_{P+1}(x_i)^2), so
// omega_i = tau^3 w_i e^{x_i} = tau^3 (P+2)/(P+1) x_i (e^{x_i/2} / L^(2)_{P+1}(x_i))^2 and
// K_p(r_i) = tau^(-3/2) e^{-x_i/2} L^(2)_p(x_i) / sqrt((p+1)(p+2)): every factor stays inside
// the float64 range for P <= 256, so no logarithms are needed.
#include <algorithm>
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "s2w_internal.h"

namespace s2w {
cudaError_t launch_radial(const double* R, const float2* R2, const double2* in, double2* out, int B, int P,
                          int64_t ncol, bool c32, cudaStream_t st);
}

struct s2w_ball_plan {
  s2w_ball_params p{};
  s2w_plan* sphere = nullptr;      // spin SHT of batch * P maps
  int Mc = 0;
  bool c32 = true;
  std::vector<double> r, omega;    // nodes and radial weights (host)
  double* Rf = nullptr;            // [P][P] omega_i K_p(r_i), row p
  double* Ri = nullptr;            // [P][P] K_p(r_i), row i
  float2* Rf2 = nullptr;
  float2* Ri2 = nullptr;
  // tensor-core precision modes (S2W_FP32_SPLIT, S2W_BF16, S2W_FP64_TC): both maps sliced for the
  // tensor cores (kernels_radx.cu) and their data-slice workspaces
  bool tc = false;
  s2w::RadxMap RfX, RiX;
  uint16_t* rops = nullptr;
  int* rfexp = nullptr;
  double2* ws = nullptr;           // [batch][P][L][Mc]
  std::vector<void*> owned;
};

namespace {

using namespace s2w;

// Double-double numbers (hi + lo, ~32 digits) for the Laguerre recurrence: in float64 the
// recurrence loses digits near the small nodes (the node error reached 1e-13 and the weight
// error 1e-11), in double-double it does not.  Built from the error-free TwoSum and
// TwoProduct (std::fma); host code is compiled with -ffp-contract=off.
struct dd {
  double hi, lo;
};
dd two_sum(double a, double b) {
  const double s = a + b, z = s - a;
  return {s, (a - (s - z)) + (b - z)};
}
dd renorm(double s, double e) {
  const double h = s + e;
  return {h, e - (h - s)};
}
dd add(dd a, dd b) {
  const dd s = two_sum(a.hi, b.hi);
  return renorm(s.hi, s.lo + a.lo + b.lo);
}
dd mul(dd a, dd b) {
  const double p = a.hi * b.hi;
  const double e = std::fma(a.hi, b.hi, -p) + (a.hi * b.lo + a.lo * b.hi);
  return renorm(p, e);
}
dd mul(dd a, double b) { return mul(a, dd{b, 0.0}); }
dd div(dd a, double b) {
  const double q1 = a.hi / b;
  const dd r = add(a, dd{-q1 * b, -std::fma(q1, b, -q1 * b)});   // a - q1*b exactly
  return renorm(q1, (r.hi + r.lo) / b);
}
dd div(dd a, dd b) {
  const double q1 = a.hi / b.hi;
  const dd r = add(a, mul(b, -q1));
  return renorm(q1, (r.hi + r.lo) / b.hi);
}

// L^(2)_0..L^(2)_{n}(x) by the three-term recurrence
// (k+1) L_{k+1} = (2k + 3 - x) L_k - (k + 2) L_{k-1}, in double-double.
void laguerre2(int n, dd x, std::vector<dd>& out) {
  out.assign(n + 1, dd{0.0, 0.0});
  out[0] = dd{1.0, 0.0};
  if (n >= 1) out[1] = add(dd{3.0, 0.0}, dd{-x.hi, -x.lo});
  for (int k = 1; k < n; ++k) {
    const dd c = add(dd{2.0 * k + 3.0, 0.0}, dd{-x.hi, -x.lo});
    out[k + 1] = div(add(mul(c, out[k]), mul(out[k - 1], -(k + 2.0))), k + 1.0);
  }
}

// number of eigenvalues of the alpha = 2 Laguerre Jacobi matrix below x (Sturm count)
int sturm_count(int P, double x) {
  int cnt = 0;
  double d = 1.0;
  for (int k = 0; k < P; ++k) {
    const double a = 2.0 * k + 3.0, b2 = (k == 0) ? 0.0 : double(k) * (k + 2.0);
    d = (a - x) - (k == 0 ? 0.0 : b2 / d);
    if (d == 0.0) d = -1e-300;
    if (d < 0.0) ++cnt;
  }
  return cnt;
}

// Roots of L^(2)_P as double-double numbers.
std::vector<dd> laguerre_nodes(int P) {
  std::vector<dd> x(P);
  const double hi = 4.0 * P + 8.0 + 4.0 * std::sqrt((double)P);   // Gershgorin bound
  std::vector<dd> L;
  for (int k = 0; k < P; ++k) {
    double lo = 0.0, up = hi;
    for (int it = 0; it < 200 && up - lo > 1e-15 * std::max(1.0, up); ++it) {
      const double mid = 0.5 * (lo + up);
      if (sturm_count(P, mid) > k) up = mid;
      else lo = mid;
    }
    dd z{0.5 * (lo + up), 0.0};
    for (int it = 0; it < 6; ++it) {   // Newton: x L_P' = P L_P - (P+2) L_{P-1}
      laguerre2(P, z, L);
      const dd d = div(add(mul(L[P], (double)P), mul(L[P - 1], -(P + 2.0))), z);
      if (d.hi == 0.0) break;
      const dd step = div(L[P], d);
      z = add(z, dd{-step.hi, -step.lo});
    }
    x[k] = z;
  }
  return x;
}

template <class T>
s2w_status up(s2w_ball_plan* B, const std::vector<T>& h, T** d, cudaStream_t st) {
  void* p = nullptr;
  if (cudaMalloc(&p, h.size() * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return record_error(S2W_ENOMEM, "cudaMalloc failed for a ball plan table");
  }
  B->owned.push_back(p);
  if (cudaMemcpyAsync(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return record_error(S2W_ECUDA, "upload of a ball plan table failed");
  *d = static_cast<T*>(p);
  return S2W_OK;
}

void destroy(s2w_ball_plan* B) {
  if (B->sphere) s2w_plan_destroy(B->sphere);
  for (void* p : B->owned) cudaFree(p);
  delete B;
}

s2w_status check_ptr(const void* p, const char* name) {
  if (p == nullptr) return record_error(S2W_EINVAL, std::string(name) + " is NULL");
  if (reinterpret_cast<uintptr_t>(p) % 8 != 0) return record_error(S2W_EINVAL, std::string(name) + " is misaligned");
  return S2W_OK;
}

int64_t ncol(const s2w_ball_plan* B) { return (int64_t)B->p.L * B->Mc; }

}  // namespace

namespace s2w {

void laguerre_rule(int P, double tau, int kmax, std::vector<double>& r, std::vector<double>& omega,
                   std::vector<double>& K) {
  const std::vector<dd> x = laguerre_nodes(P);
  std::vector<dd> Lv;
  r.assign(P, 0.0);
  omega.assign(P, 0.0);
  K.assign((size_t)P * kmax, 0.0);
  for (int i = 0; i < P; ++i) {
    laguerre2(std::max(P + 1, kmax), x[i], Lv);
    // e^{x/2} to ~1 ulp at the double-double node: e^{hi/2} (1 + lo/2)
    const double eh = std::exp(0.5 * x[i].hi) * (1.0 + 0.5 * x[i].lo);
    const dd q = div(dd{eh, 0.0}, Lv[P + 1]);
    const dd q2 = mul(mul(q, q), x[i]);
    r[i] = tau * (x[i].hi + x[i].lo);
    omega[i] = tau * tau * tau * (P + 2.0) / (P + 1.0) * (q2.hi + q2.lo);
    const double damp = 1.0 / (eh * std::pow(tau, 1.5));
    for (int k = 0; k < kmax; ++k)
      K[(size_t)i * kmax + k] = damp * (Lv[k].hi + Lv[k].lo) / std::sqrt((k + 1.0) * (k + 2.0));
  }
}

}  // namespace s2w

using namespace s2w;

extern "C" {

s2w_status s2w_ball_plan_create(const s2w_ball_params* prm, void* stream, s2w_ball_plan** out) {
  if (out == nullptr) return record_error(S2W_EINVAL, "out is NULL");
  *out = nullptr;
  if (prm == nullptr) return record_error(S2W_EINVAL, "params is NULL");
  const s2w_ball_params p = *prm;
  if (p.P < 2 || p.P > 256) return record_error(S2W_EINVAL, "P must satisfy 2 <= P <= 256");
  if (!(p.tau > 0.0) || !std::isfinite(p.tau)) return record_error(S2W_EINVAL, "tau must be > 0");
  if (p.batch < 1) return record_error(S2W_EINVAL, "batch must be >= 1");
  if (p.precision < S2W_FP64 || p.precision > S2W_FP64_TC) return record_error(S2W_EINVAL, "unknown precision mode");
  s2w_ball_plan* B = new (std::nothrow) s2w_ball_plan();
  if (B == nullptr) return record_error(S2W_ENOMEM, "host allocation failed");
  B->p = p;
  B->c32 = p.precision != S2W_FP64_NATIVE;
  B->tc = p.precision == S2W_FP32_SPLIT || p.precision == S2W_BF16 || p.precision == S2W_FP64_TC;
  s2w_params sp{};
  sp.L = p.L;
  sp.N = 1;
  sp.J0 = 0;
  sp.spin = p.spin;
  sp.reality = p.reality;
  sp.batch = p.batch * p.P;
  sp.precision = p.precision;
  sp.precompute = 0;
  sp.lambda = 2.0;
  sp.sampling = p.sampling;
  s2w_status s = s2w_plan_create(&sp, stream, &B->sphere);   // validates L, spin, reality
  if (s != S2W_OK) {
    delete B;
    return s;
  }
  // the radial maps amplify the sphere transforms' error about a hundredfold: in S2W_FP64_TC the
  // sliced GEMMs of this plan also sum the digit-pair diagonal 7
  B->sphere->slice_diag7 = 1;
  B->Mc = p.reality ? p.L : 2 * p.L - 1;
  const int P = p.P;
  const double tau = p.tau;
  std::vector<double> Rf((size_t)P * P), Ri((size_t)P * P), Kt;
  laguerre_rule(P, tau, P, B->r, B->omega, Kt);
  for (int i = 0; i < P; ++i)
    for (int k = 0; k < P; ++k) {
      const double K = Kt[(size_t)i * P + k];   // K_k(r_i)
      Rf[(size_t)k * P + i] = B->omega[i] * K;
      Ri[(size_t)i * P + k] = K;
    }
  std::vector<float2> Rf2(Rf.size()), Ri2(Ri.size());
  for (size_t k = 0; k < Rf.size(); ++k) {
    float h = (float)Rf[k];
    Rf2[k] = make_float2(h, (float)(Rf[k] - (double)h));
    h = (float)Ri[k];
    Ri2[k] = make_float2(h, (float)(Ri[k] - (double)h));
  }
  cudaStream_t st = (cudaStream_t)stream;
  if ((s = up(B, Rf, &B->Rf, st)) || (s = up(B, Ri, &B->Ri, st)) || (s = up(B, Rf2, &B->Rf2, st)) ||
      (s = up(B, Ri2, &B->Ri2, st))) {
    destroy(B);
    return s;
  }
  if (B->tc) {
    // Rf as stored is [p][i] (row p); Ri is [i][p]: the inverse map f_r[i] = sum_p K_p(r_i) f_p[p]
    // has rows i, so its matrix is Ri itself
    std::vector<uint16_t> tab;
    std::vector<int> rexp, kexp;
    build_radx(Rf, P, P, &B->RfX, tab, rexp, kexp);
    if ((s = up(B, tab, &B->RfX.tab, st)) || (s = up(B, rexp, &B->RfX.rexp, st)) || (s = up(B, kexp, &B->RfX.kexp, st)))
      return destroy(B), s;
    build_radx(Ri, P, P, &B->RiX, tab, rexp, kexp);
    if ((s = up(B, tab, &B->RiX.tab, st)) || (s = up(B, rexp, &B->RiX.rexp, st)) || (s = up(B, kexp, &B->RiX.kexp, st)))
      return destroy(B), s;
    std::vector<uint16_t> ops((size_t)radx_ops_elems(p.batch, P, ncol(B)), 0);
    std::vector<int> fx((size_t)p.batch * ncol(B) * 2, 0);
    if ((s = up(B, ops, &B->rops, st)) || (s = up(B, fx, &B->rfexp, st))) return destroy(B), s;
  }
  void* w = nullptr;
  if (cudaMalloc(&w, (size_t)p.batch * P * ncol(B) * sizeof(double2)) != cudaSuccess) {
    cudaGetLastError();
    destroy(B);
    return record_error(S2W_ENOMEM, "ball workspace allocation failed");
  }
  B->owned.push_back(w);
  B->ws = static_cast<double2*>(w);
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    destroy(B);
    return record_error(S2W_ECUDA, "ball plan upload failed");
  }
  *out = B;
  return S2W_OK;
}

s2w_status s2w_ball_plan_destroy(s2w_ball_plan* B) {
  if (B == nullptr) return record_error(S2W_EINVAL, "plan is NULL");
  destroy(B);
  return S2W_OK;
}

s2w_status s2w_ball_nodes(const s2w_ball_plan* B, double* r, double* omega) {
  if (B == nullptr) return record_error(S2W_EINVAL, "plan is NULL");
  for (int i = 0; i < B->p.P; ++i) {
    if (r) r[i] = B->r[i];
    if (omega) omega[i] = B->omega[i];
  }
  return S2W_OK;
}

s2w_status s2w_laguerre_forward(const s2w_ball_plan* B, const void* f_r, void* f_p, void* stream) {
  if (B == nullptr) return record_error(S2W_EINVAL, "plan is NULL");
  s2w_status s;
  if ((s = check_ptr(f_r, "f_r")) || (s = check_ptr(f_p, "f_p"))) return s;
  cudaError_t e =
      B->tc ? launch_radx(B->RfX, (const double2*)f_r, (double2*)f_p, B->p.batch, B->p.L, B->Mc, nullptr, nullptr,
                          false, B->rops, B->rfexp, B->sphere->err_word, (cudaStream_t)stream)
            : launch_radial(B->Rf, B->Rf2, (const double2*)f_r, (double2*)f_p, B->p.batch, B->p.P, ncol(B), B->c32,
                            (cudaStream_t)stream);
  if (e != cudaSuccess) return record_error(S2W_ECUDA, std::string("radial transform: ") + cudaGetErrorString(e));
  return S2W_OK;
}

s2w_status s2w_laguerre_inverse(const s2w_ball_plan* B, const void* f_p, void* f_r, void* stream) {
  if (B == nullptr) return record_error(S2W_EINVAL, "plan is NULL");
  s2w_status s;
  if ((s = check_ptr(f_p, "f_p")) || (s = check_ptr(f_r, "f_r"))) return s;
  cudaError_t e =
      B->tc ? launch_radx(B->RiX, (const double2*)f_p, (double2*)f_r, B->p.batch, B->p.L, B->Mc, nullptr, nullptr,
                          false, B->rops, B->rfexp, B->sphere->err_word, (cudaStream_t)stream)
            : launch_radial(B->Ri, B->Ri2, (const double2*)f_p, (double2*)f_r, B->p.batch, B->p.P, ncol(B), B->c32,
                            (cudaStream_t)stream);
  if (e != cudaSuccess) return record_error(S2W_ECUDA, std::string("radial transform: ") + cudaGetErrorString(e));
  return S2W_OK;
}

s2w_status s2w_ball_sl_forward(const s2w_ball_plan* B, const void* f, void* flmp, void* stream) {
  if (B == nullptr) return record_error(S2W_EINVAL, "plan is NULL");
  s2w_status s;
  if ((s = check_ptr(flmp, "flmp"))) return s;
  if ((s = s2w_sht_forward(B->sphere, f, B->ws, stream))) return s;
  return s2w_laguerre_forward(B, B->ws, flmp, stream);
}

s2w_status s2w_ball_sl_inverse(const s2w_ball_plan* B, const void* flmp, void* f, void* stream) {
  if (B == nullptr) return record_error(S2W_EINVAL, "plan is NULL");
  s2w_status s;
  if ((s = s2w_laguerre_inverse(B, flmp, B->ws, stream))) return s;
  return s2w_sht_inverse(B->sphere, B->ws, f, stream);
}

}  // extern "C"
