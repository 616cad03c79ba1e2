// Host-side construction of a transform plan: parameter validation, the wavelet
// dictionary (App. A), multiresolution band-limits (Sec. 3.3), and the float64
// tables the kernels read (MW or DH grids, Wigner-d seed powers, the colatitude
// quadrature: MW matrices or DH ring weights, and DFT twiddles).  Everything here runs
// once per plan.
#include <cmath>
#include <complex>
#include <cstring>
#include <map>
#include <numeric>
#include <tuple>

#include "s2w_internal.h"
#include "tiling.h"

namespace s2w {
namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;
using cplx = std::complex<double>;
using tiling::Tiling;
using tiling::ceil_pow;

// Azimuthal tiling zeta_lm (Eq. A6).
cplx zeta(int l, int m, int N) {
  bool mu = ((N + m) % 2 + 2) % 2 == 1;
  int q = std::min(N - 1, l - (((N + l) % 2 == 0) ? 1 : 0));
  if (!mu || q < 0 || std::abs(m) > q || ((q - m) % 2) != 0) return 0.0;
  int k = (q - m) / 2;
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r *= double(q - k + i) / double(i);
  r = std::ldexp(r, -q);
  double v = std::sqrt(r);
  return ((N - 1) % 2 == 0) ? cplx(v, 0.0) : cplx(0.0, v);
}

// ---------------------------------------------------------------- grids

// exp(-i p theta_u), theta_u = pi (2u+1)/n, with exact integer argument reduction.
cplx phase_theta(long p, long u, long n) {
  long num = ((p * (2 * u + 1)) % (2 * n) + 2 * n) % (2 * n);
  double a = kPi * double(num) / double(n);
  return cplx(std::cos(a), -std::sin(a));
}

double sin_weight_re(long q) { return (q % 2 == 0) ? 2.0 / (1.0 - double(q) * double(q)) : 0.0; }
double sin_weight_im(long q) { return q == 1 ? 0.5 * kPi : (q == -1 ? -0.5 * kPi : 0.0); }

// Colatitude quadrature matrix for parity sigma (= (-1)^(m+n)): Mq[t][t'] such that
// int_0^pi G(theta) d(theta) sin(theta) d theta = sum_t (Mq G)_t d(theta_t) for every
// column G and Wigner function d of that parity band-limited at L (MW sampling).
// Built column by column from the extend / DFT / sin-weight convolution / inverse
// DFT / fold steps applied to unit impulses.
void quad_matrix(int L, int sigma, std::vector<double>& M /* [t][t'] */) {
  const long n = 2 * L - 1;
  M.assign((size_t)L * L, 0.0);
  std::vector<cplx> X(n), H(n), g(n);
  // w(p + q) for p, q in [-(L-1), L-1]
  for (int tp = 0; tp < L; ++tp) {
    // Fourier coefficients of the parity-extended impulse at theta_tp.
    for (long p = -(L - 1); p <= L - 1; ++p) {
      cplx v = phase_theta(p, tp, n);
      if (tp < L - 1) v += double(sigma) * phase_theta(p, n - 1 - tp, n);
      X[p + L - 1] = v / double(n);
    }
    for (long q = -(L - 1); q <= L - 1; ++q) {
      cplx acc = 0.0;
      for (long p = -(L - 1); p <= L - 1; ++p) {
        long k = p + q;
        double wr = sin_weight_re(k), wi = sin_weight_im(k);
        if (wr == 0.0 && wi == 0.0) continue;
        acc += X[p + L - 1] * cplx(wr, wi);
      }
      H[q + L - 1] = acc;
    }
    for (long u = 0; u < n; ++u) {
      cplx acc = 0.0;
      for (long q = -(L - 1); q <= L - 1; ++q) acc += H[q + L - 1] * phase_theta(q, u, n);
      g[u] = acc / double(n);
    }
    for (int t = 0; t < L; ++t) {
      cplx v = g[t];
      if (t < L - 1) v += double(sigma) * g[n - 1 - t];
      M[(size_t)t * L + tp] = v.real();
    }
  }
}

template <class T>
s2w_status upload(s2w_plan* P, const std::vector<T>& h, T** d, cudaStream_t st, std::string& err) {
  *d = nullptr;
  if (h.empty()) return S2W_OK;
  void* p = nullptr;
  if (cudaMalloc(&p, h.size() * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    err = "cudaMalloc failed for a plan table";
    return S2W_ENOMEM;
  }
  P->owned.push_back(p);
  P->owned_bytes.push_back(h.size() * sizeof(T));
  if (cudaMemcpyAsync(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, st) != cudaSuccess) {
    err = "cudaMemcpyAsync failed while uploading a plan table";
    return S2W_ECUDA;
  }
  *d = static_cast<T*>(p);
  return S2W_OK;
}

#define S2W_TRY(x)                   \
  do {                               \
    s2w_status _s = (x);             \
    if (_s != S2W_OK) return _s;     \
  } while (0)

// float64 complex -> (re_hi, re_lo, im_hi, im_lo) float pair representation
float4 split4(double2 v) {
  float rh = (float)v.x, ih = (float)v.y;
  return make_float4(rh, (float)(v.x - (double)rh), ih, (float)(v.y - (double)ih));
}

void factorise(int n, int& n1, int& n2) {
  n1 = 1;
  n2 = n;
  for (int a = 2; a * a <= n; ++a)
    if (n % a == 0) {
      n1 = a;
      n2 = n / a;
    }
}

// Driscoll-Healy ring weights on the 2L midpoint rings theta_t = pi (2t+1)/(4L):
//   w_t = (2/L) sin(theta_t) sum_{k<L} sin((2k+1) theta_t)/(2k+1),
// the unique weights that integrate cos(j theta) sin(theta) over [0, pi] exactly for j < 2L
// (the Driscoll-Healy quadrature; Fejer's first rule in x = cos theta).  Every sine has an
// integer multiple of pi/(4L) as argument, reduced exactly before evaluation.
std::vector<double> dh_weights(int L) {
  const long den = 4L * L;   // angles pi a/den
  auto sin_pi = [&](long a) {
    a %= 2 * den;
    if (a < 0) a += 2 * den;
    const double sg = (a >= den) ? -1.0 : 1.0;
    if (a >= den) a -= den;
    if (2 * a > den) a = den - a;   // sin(pi - x) = sin x
    return sg * std::sin(kPi * double(a) / double(den));
  };
  std::vector<double> w(2 * L);
  for (int t = 0; t < 2 * L; ++t) {
    long double acc = 0.0L;
    for (int k = 0; k < L; ++k) acc += (long double)sin_pi((long)(2 * k + 1) * (2 * t + 1)) / (long double)(2 * k + 1);
    w[t] = (double)((2.0L / (long double)L) * (long double)sin_pi(2 * t + 1) * acc);
  }
  return w;
}

s2w_status build_grid(s2w_plan* P, int L, cudaStream_t st, GridTables& g, std::string& err) {
  const bool dh = P->p.sampling == S2W_SAMPLING_DH;
  g.L = L;
  g.n = 2 * L - 1;
  g.nr = rings_of(P->p.sampling, L);
  g.den = dh ? 4 * L : g.n;
  factorise(g.n, g.n1, g.n2);
  const int n = g.n, nr = g.nr, den = g.den;
  std::vector<double> wpole(nr), cm((size_t)nr * n), sm((size_t)nr * n), sc((size_t)L * n, 0.0);
  std::vector<int> ce((size_t)nr * n), se((size_t)nr * n);
  for (int b = 0; b < nr; ++b) {
    // half angle beta_b/2 = pi num/(2 den); the smaller of sin and cos is evaluated through an
    // exact complementary argument so both keep full relative precision near the poles.
    const long num = 2 * b + 1, cnum = den - num;   // pi/2 - beta_b/2 = pi cnum/(2 den)
    double ch, sh;
    if (2 * num <= den) {
      sh = std::sin(0.5 * kPi * double(num) / double(den));
      ch = std::cos(0.5 * kPi * double(num) / double(den));
    } else {
      ch = (cnum == 0) ? 0.0 : std::sin(0.5 * kPi * double(cnum) / double(den));
      sh = (cnum == 0) ? 1.0 : std::cos(0.5 * kPi * double(cnum) / double(den));
    }
    // recursion weight: -(1 - cos beta) = -2 sin^2(beta/2) on the northern half,
    // (1 + cos beta) = 2 cos^2(beta/2) on the southern half (see rec_coeffs).
    wpole[b] = (2 * num < den) ? -2.0 * sh * sh : 2.0 * ch * ch;
    // powers as (mantissa in [0.5,1), exponent); zero base gives exact zeros.
    double vm = 0.5, sv = 0.5;
    int ve = 1, svx = 1;
    for (int a = 0; a < n; ++a) {
      cm[(size_t)b * n + a] = vm;
      ce[(size_t)b * n + a] = ve;
      sm[(size_t)b * n + a] = sv;
      se[(size_t)b * n + a] = svx;
      int d;
      vm = std::frexp(vm * ch, &d);
      ve = (vm == 0.0) ? 0 : ve + d;
      sv = std::frexp(sv * sh, &d);
      svx = (sv == 0.0) ? 0 : svx + d;
    }
  }
  for (int l = 0; l < L; ++l) {
    double v = 1.0;
    sc[(size_t)l * n] = 1.0;
    for (int k = 1; k <= 2 * l; ++k) {
      v *= std::sqrt(double(2 * l - k + 1) / double(k));
      sc[(size_t)l * n + k] = v;
    }
  }
  std::vector<double2> tw(n);
  std::vector<float4> tw4(n);
  for (int e = 0; e < n; ++e) {
    double a = 2.0 * kPi * double(e) / double(n);
    tw[e] = make_double2(std::cos(a), std::sin(a));
    tw4[e] = split4(tw[e]);
  }
  S2W_TRY(upload(P, wpole, &g.wpole, st, err));
  S2W_TRY(upload(P, cm, &g.cpow_m, st, err));
  S2W_TRY(upload(P, ce, &g.cpow_e, st, err));
  S2W_TRY(upload(P, sm, &g.spow_m, st, err));
  S2W_TRY(upload(P, se, &g.spow_e, st, err));
  S2W_TRY(upload(P, sc, &g.sqrtC, st, err));
  if (dh) {
    S2W_TRY(upload(P, dh_weights(L), &g.wdiag, st, err));
  } else {
    std::vector<double> MT((size_t)2 * L * L), M;
    for (int par = 0; par < 2; ++par) {
      quad_matrix(L, par == 0 ? 1 : -1, M);
      for (int t = 0; t < L; ++t)
        for (int tp = 0; tp < L; ++tp) MT[(size_t)par * L * L + (size_t)tp * L + t] = M[(size_t)t * L + tp];
    }
    std::vector<float2> MT2(MT.size()), MR2(MT.size());
    std::vector<double> MR(MT.size());
    for (int par = 0; par < 2; ++par)
      for (int t = 0; t < L; ++t)
        for (int tp = 0; tp < L; ++tp)
          MR[(size_t)par * L * L + (size_t)t * L + tp] = MT[(size_t)par * L * L + (size_t)tp * L + t];
    for (size_t i = 0; i < MT.size(); ++i) {
      float h = (float)MT[i];
      MT2[i] = make_float2(h, (float)(MT[i] - (double)h));
      h = (float)MR[i];
      MR2[i] = make_float2(h, (float)(MR[i] - (double)h));
    }
    S2W_TRY(upload(P, MT, &g.MT, st, err));
    S2W_TRY(upload(P, MT2, &g.MT2, st, err));
    S2W_TRY(upload(P, MR, &g.MR, st, err));
    S2W_TRY(upload(P, MR2, &g.MR2, st, err));
  }
  S2W_TRY(upload(P, tw, &g.tw, st, err));
  S2W_TRY(upload(P, tw4, &g.tw4, st, err));
  return S2W_OK;
}

s2w_status build_spec(s2w_plan* P, cudaStream_t st, TransformSpec& t, int L, int N, int grid,
                      const std::vector<int>& nvals, const std::vector<cplx>& minv,
                      const std::vector<cplx>& mfwd, double gscale, std::string& err) {
  t.L = L;
  t.N = N;
  t.grid = grid;
  t.nact = (int)nvals.size();
  t.nvals_h = nvals;
  std::vector<double2> a(minv.size()), b(mfwd.size()), ph((size_t)t.nact * (2 * N - 1));
  std::vector<float4> ph4(ph.size());
  for (size_t i = 0; i < minv.size(); ++i) a[i] = make_double2(minv[i].real(), minv[i].imag());
  for (size_t i = 0; i < mfwd.size(); ++i) b[i] = make_double2(mfwd[i].real(), mfwd[i].imag());
  const long ng = 2 * N - 1;
  for (int i = 0; i < t.nact; ++i)
    for (long gi = 0; gi < ng; ++gi) {
      long num = ((long)nvals[i] * gi % ng + ng) % ng;
      double ang = 2.0 * kPi * double(num) / double(ng);
      ph[(size_t)i * ng + gi] = make_double2(std::cos(ang), std::sin(ang));
      ph4[(size_t)i * ng + gi] = split4(ph[(size_t)i * ng + gi]);
    }
  t.gscale = gscale;
  // the l-contractions only need l where some multiplier is nonzero (the wavelet filters
  // vanish below their scale's support, Eq. A3)
  t.lmin_h = L;
  for (int l = 0; l < L && t.lmin_h == L; ++l)
    for (int i = 0; i < t.nact; ++i)
      if (minv[(size_t)l * t.nact + i] != cplx(0.0) || mfwd[(size_t)l * t.nact + i] != cplx(0.0)) {
        t.lmin_h = l;
        break;
      }
  // adjoint multipliers: the forward DFT kernel carries (2 pi/(2L-1)) gscale, the inverse
  // none, so transposing a DFT moves that factor into the contraction beside it.
  const double dft_scale = (2.0 * kPi / (2.0 * L - 1.0)) * gscale;
  std::vector<double2> af(minv.size()), ai(mfwd.size());
  for (size_t i = 0; i < minv.size(); ++i)
    af[i] = make_double2(minv[i].real() / dft_scale, -minv[i].imag() / dft_scale);
  for (size_t i = 0; i < mfwd.size(); ++i)
    ai[i] = make_double2(mfwd[i].real() * dft_scale, -mfwd[i].imag() * dft_scale);
  {
    // factor mult_inv into one complex phase times real values, when it has that form
    size_t imax = 0;
    double amax = 0.0;
    for (size_t i = 0; i < minv.size(); ++i)
      if (std::abs(minv[i]) > amax) amax = std::abs(minv[i]), imax = i;
    const cplx ph = amax > 0.0 ? minv[imax] / amax : cplx(1.0, 0.0);
    std::vector<double> r(minv.size());
    bool ok = true;
    for (size_t i = 0; i < minv.size(); ++i) {
      const cplx q = minv[i] * std::conj(ph);
      r[i] = q.real();
      if (std::abs(q.imag()) > 1e-15 * amax) ok = false;
    }
    t.minv_phase = make_double2(ph.real(), ph.imag());
    t.minv_factored = ok;
    S2W_TRY(upload(P, r, &t.minv_r, st, err));
  }
  S2W_TRY(upload(P, af, &t.adj_fwd, st, err));
  S2W_TRY(upload(P, ai, &t.adj_inv, st, err));
  S2W_TRY(upload(P, nvals, &t.nvals, st, err));
  S2W_TRY(upload(P, a, &t.mult_inv, st, err));
  S2W_TRY(upload(P, b, &t.mult_fwd, st, err));
  S2W_TRY(upload(P, ph, &t.gphase, st, err));
  S2W_TRY(upload(P, ph4, &t.gphase4, st, err));
  return S2W_OK;
}

// Workspace (per-call scratch sized for the batch, as opposed to the plan's tables): counted in
// P->workspace_bytes for s2w_plan_device_bytes.
template <class T>
s2w_status alloc_ws(s2w_plan* P, size_t n, T** d, std::string& err) {
  void* q = nullptr;
  if (cudaMalloc(&q, n * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    err = "workspace allocation failed";
    return S2W_ENOMEM;
  }
  P->owned.push_back(q);
  P->owned_bytes.push_back(n * sizeof(T));
  P->workspace_bytes += (int64_t)(n * sizeof(T));
  *d = static_cast<T*>(q);
  return S2W_OK;
}

template <class T>
s2w_status alloc_dev(s2w_plan* P, size_t n, T** d, std::string& err) {
  void* q = nullptr;
  if (cudaMalloc(&q, n * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    err = "device allocation of the packed Wigner-d tables failed";
    return S2W_ENOMEM;
  }
  P->owned.push_back(q);
  P->owned_bytes.push_back(n * sizeof(T));
  *d = static_cast<T*>(q);
  return S2W_OK;
}

// Reduced-precision modes: packed Wigner-d tiles for the wavelet-scale Wigner transforms
// (cached per band-limit and n set, so scales with equal (L_j, N_j) share them) and packed
// quadrature matrices.  The spin SHT and the scaling transform stay float64-accurate (the
// sliced tensor-core kernels): Y f sets the accuracy of every small high-l coefficient the top
// scales see, and with a steep spectrum a 16-bit quantisation relative to f_00 would swamp them.
s2w_status make_tab(s2w_plan* P, const TransformSpec& t, TabTable* tab, cudaStream_t st, std::string& err);

// Tensor-core tables of the reduced modes for every wavelet scale (specs with the same (L, n
// values) share one), packed from temporary float-pair tables (make_tab: float64 recursion and
// the folded quadrature) that are freed once packed; plus the operand workspace.
s2w_status build_tc_tables(s2w_plan* P, cudaStream_t st, std::string& err) {
  const bool fp16 = P->p.precision == S2W_FP32_SPLIT;
  std::map<std::pair<int, std::vector<int>>, TcTable*> cache;
  int64_t op_max = 0, sc_max = 0;
  const int nq = (P->p.batch + 15) / 16;
  for (TransformSpec& tr : P->wav_t) {
    TransformSpec* t = &tr;
    auto key = std::make_pair(t->L, t->nvals_h);
    auto it = cache.find(key);
    if (it != cache.end()) {
      t->tc = it->second;
      continue;
    }
    const int L = t->L, Mc = P->real ? L : 2 * L - 1, mlo = P->real ? 0 : -(L - 1);
    const int nr = rings_of(P->p.sampling, L);
    TcTable* tab = new TcTable();
    P->tc_tables.push_back(tab);
    tab->Lb = ((nr + 127) / 128) * 128;
    tab->Lk = ((nr + 63) / 64) * 64;
    std::vector<int64_t> oi((size_t)Mc * t->nact, 0), of((size_t)Mc * t->nact, 0);
    std::vector<int> ki((size_t)Mc * t->nact, 0), kf((size_t)Mc * t->nact, 0);
    int64_t ri = 0, rf = 0;
    for (int mi = 0; mi < Mc; ++mi)
      for (int ni = 0; ni < t->nact; ++ni) {
        const size_t idx = (size_t)mi * t->nact + ni;
        const int l0 = std::max(std::abs(mlo + mi), std::abs(t->nvals_h[ni]));
        oi[idx] = ri;
        of[idx] = rf;
        if (l0 >= L) continue;
        const int l0a = l0 & ~7;
        ki[idx] = ((L - l0a + 63) / 64) * 64;
        kf[idx] = ((L - l0a + 127) / 128) * 128;
        ri += (int64_t)tab->Lb * ki[idx];
        rf += (int64_t)kf[idx] * tab->Lk;
        tab->klf_max = std::max(tab->klf_max, kf[idx]);
      }
    tab->op_i = 32 * (ri / tab->Lb);
    tab->op_f = 32 * (int64_t)tab->Lk * Mc * t->nact;
    op_max = std::max(op_max, std::max(tab->op_i, tab->op_f));
    sc_max = std::max(sc_max, (int64_t)Mc * t->nact);
    S2W_TRY(upload(P, oi, &tab->off_i, st, err));
    S2W_TRY(upload(P, of, &tab->off_f, st, err));
    S2W_TRY(upload(P, ki, &tab->kli, st, err));
    S2W_TRY(upload(P, kf, &tab->klf, st, err));
    S2W_TRY(alloc_dev(P, (size_t)std::max<int64_t>(ri, 1), &tab->inv_hi, err));
    S2W_TRY(alloc_dev(P, (size_t)std::max<int64_t>(ri, 1), &tab->inv_lo, err));
    S2W_TRY(alloc_dev(P, (size_t)std::max<int64_t>(rf, 1), &tab->fwd_hi, err));
    S2W_TRY(alloc_dev(P, (size_t)std::max<int64_t>(rf, 1), &tab->fwd_lo, err));
    // temporary float-pair tables: their allocations are the ones added to P->owned here
    const size_t mark = P->owned.size();
    TabTable tmp;
    S2W_TRY(make_tab(P, *t, &tmp, st, err));
    if (launch_tc_pack(*t, *tab, tmp, nr, Mc, mlo, fp16, st) != cudaSuccess) {
      err = "tensor-core table packing failed to launch";
      return S2W_ECUDA;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) {
      err = "tensor-core table build failed";
      return S2W_ECUDA;
    }
    for (size_t i = mark; i < P->owned.size(); ++i) cudaFree(P->owned[i]);
    P->owned.resize(mark);
    P->owned_bytes.resize(mark);
    cache[key] = tab;
    t->tc = tab;
  }
  S2W_TRY(alloc_ws(P, (size_t)std::max<int64_t>(nq * op_max, 1), &P->tc_b_hi, err));
  S2W_TRY(alloc_ws(P, (size_t)std::max<int64_t>(nq * op_max, 1), &P->tc_b_lo, err));
  S2W_TRY(alloc_ws(P, (size_t)std::max<int64_t>(nq * sc_max, 1), &P->tc_scale, err));
  return S2W_OK;
}

// Sliced tables for the SHT, the scaling function and (S2W_FP64_TC: with_wavelets) the wavelet
// scales; specs with the same (L, n values) share one.  Packed from temporary float-pair tables
// (make_tab) that are freed once packed; plus the data-slice workspace.
s2w_status build_tcx_tables(s2w_plan* P, cudaStream_t st, std::string& err, bool with_wavelets) {
  std::map<std::tuple<int, std::vector<int>, int>, TcxTable*> cache;
  std::vector<TransformSpec*> specs = {&P->sht, &P->scal_t};
  if (with_wavelets)
    for (TransformSpec& t : P->wav_t) specs.push_back(&t);
  int64_t op_max = 0, fx_max = 0;
  const int nq = (P->p.batch + 15) / 16;
  for (TransformSpec* t : specs) {
    auto key = std::make_tuple(t->L, t->nvals_h, t->lmin_h);
    auto it = cache.find(key);
    if (it != cache.end()) {
      t->tcx = it->second;
      continue;
    }
    const int L = t->L, Mc = P->real ? L : 2 * L - 1, mlo = P->real ? 0 : -(L - 1);
    const int nr = rings_of(P->p.sampling, L);
    TcxTable* tab = new TcxTable();
    P->tcx_tables.push_back(tab);
    tab->lmin = t->lmin_h;
    tab->Lb = ((nr + 127) / 128) * 128;
    tab->Lk = ((nr + 15) / 16) * 16;
    const size_t nidx = (size_t)Mc * t->nact;
    std::vector<int64_t> oi(nidx, 0), of(nidx, 0), oo(nidx, 0);
    std::vector<int> ki(nidx, 0), kf(nidx, 0);
    int64_t ri = 0, rf = 0, ro = 0;
    for (int mi = 0; mi < Mc; ++mi)
      for (int ni = 0; ni < t->nact; ++ni) {
        const size_t idx = (size_t)mi * t->nact + ni;
        const int l0 = std::max(std::max(std::abs(mlo + mi), std::abs(t->nvals_h[ni])), t->lmin_h);
        oi[idx] = ri;
        of[idx] = rf;
        oo[idx] = ro;
        if (l0 >= L) continue;
        const int l0a = l0 & ~7;
        ki[idx] = ((L - l0a + 15) / 16) * 16;
        kf[idx] = ((L - l0a + 127) / 128) * 128;
        ri += (int64_t)tab->Lb * ki[idx] * 7;
        rf += (int64_t)kf[idx] * tab->Lk * 7;
        ro += (int64_t)32 * 7 * ki[idx];
        tab->klf_max = std::max(tab->klf_max, kf[idx]);
        tab->kli_max = std::max(tab->kli_max, ki[idx]);
      }
    tab->op_i = ro;
    tab->op_f = (int64_t)32 * 7 * tab->Lk * (int64_t)nidx;
    op_max = std::max(op_max, std::max(tab->op_i, tab->op_f));
    fx_max = std::max<int64_t>(fx_max, (int64_t)nidx * 32);
    S2W_TRY(upload(P, oi, &tab->off_i, st, err));
    S2W_TRY(upload(P, of, &tab->off_f, st, err));
    S2W_TRY(upload(P, oo, &tab->opoff_i, st, err));
    S2W_TRY(upload(P, ki, &tab->kli, st, err));
    S2W_TRY(upload(P, kf, &tab->klf, st, err));
    S2W_TRY(alloc_dev(P, std::max<size_t>(nidx * tab->Lb, 1), &tab->rexp_i, err));
    S2W_TRY(alloc_dev(P, std::max<size_t>(nidx * (size_t)tab->klf_max, 1), &tab->rexp_f, err));
    S2W_TRY(alloc_dev(P, (size_t)std::max<int64_t>(ri, 1), &tab->inv, err));
    S2W_TRY(alloc_dev(P, (size_t)std::max<int64_t>(rf, 1), &tab->fwd, err));
    const size_t mark = P->owned.size();
    TabTable tmp;
    S2W_TRY(make_tab(P, *t, &tmp, st, err));
    if (tmp.kpmax > 0 && launch_tcx_pack(*t, *tab, tmp, nr, Mc, mlo, st) != cudaSuccess) {
      err = "sliced table packing failed to launch";
      return S2W_ECUDA;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) {
      err = "sliced table build failed";
      return S2W_ECUDA;
    }
    for (size_t i = mark; i < P->owned.size(); ++i) cudaFree(P->owned[i]);
    P->owned.resize(mark);
    P->owned_bytes.resize(mark);
    cache[key] = tab;
    t->tcx = tab;
  }
  S2W_TRY(alloc_ws(P, (size_t)std::max<int64_t>(nq * op_max, 1), &P->tcx_ops, err));
  S2W_TRY(alloc_ws(P, (size_t)std::max<int64_t>(nq * fx_max, 1), &P->tcx_fexp, err));
  return S2W_OK;
}

// Sliced twiddle tables of the tensor-core DFTs for the SHT, the scaling function and
// (S2W_FP64_TC: with_wavelets) the wavelet scales and raw Wigner transforms, where the carried n
// values fit (dftx_shape_ok): per band-limit one inverse table (scale 1) and one forward table
// per normalisation (2 pi/(2L-1)) gscale, shared between specs; plus the data-slice workspace.
s2w_status build_dftx_tables(s2w_plan* P, cudaStream_t st, std::string& err, bool with_wavelets) {
  std::map<std::pair<int, double>, DftxTable*> cache;
  std::vector<TransformSpec*> specs = {&P->sht, &P->scal_t};
  if (with_wavelets) {
    for (TransformSpec& t : P->wav_t) specs.push_back(&t);
    for (TransformSpec& t : P->raw_t) specs.push_back(&t);
  }
  int64_t ops = 0, fx = 0;
  auto table = [&](int L, double scale, const DftxTable** out) -> s2w_status {
    auto key = std::make_pair(L, scale);
    auto it = cache.find(key);
    if (it != cache.end()) {
      *out = it->second;
      return S2W_OK;
    }
    DftxTable* tab = new DftxTable();
    P->dftx_tables.push_back(tab);
    std::vector<uint16_t> hc, hs;
    build_dftx_table(L, scale, tab, hc, hs);
    S2W_TRY(upload(P, hc, &tab->cos, st, err));
    S2W_TRY(upload(P, hs, &tab->sin, st, err));
    cache[key] = tab;
    *out = tab;
    return S2W_OK;
  };
  // prime-factor tables (kernels_dftp.cu), per (L, n1, normalisation)
  std::map<std::tuple<int, int, double>, DftpTable*> pcache;
  auto ptable = [&](int L, int n1, int n2, double scale, const DftpTable** out) -> s2w_status {
    auto key = std::make_tuple(L, n1, scale);
    auto it = pcache.find(key);
    if (it != pcache.end()) {
      *out = it->second;
      return S2W_OK;
    }
    DftpTable* tab = new DftpTable();
    P->dftp_tables.push_back(tab);
    std::vector<uint16_t> h;
    build_dftp_table(L, n1, n2, scale, tab, h);
    S2W_TRY(upload(P, h, &tab->tab, st, err));
    pcache[key] = tab;
    *out = tab;
    return S2W_OK;
  };
  int64_t pops = 0, pfx = 0, pz = 0;
  for (TransformSpec* t : specs) {
    int n1 = 0, n2 = 0;
    if (dftp_shape(*t, P->real, &n1, &n2)) {
      S2W_TRY(ptable(t->L, n1, n2, 1.0, &t->dftp_inv));
      S2W_TRY(ptable(t->L, n1, n2, (2.0 * kPi / (2.0 * t->L - 1.0)) * t->gscale, &t->dftp_fwd));
      int64_t o = 0, f = 0, z = 0;
      dftp_ws_elems(*t, P->real, n1, P->p.batch, rings_of(P->p.sampling, t->L), &o, &f, &z);
      pops = std::max(pops, o);
      pfx = std::max(pfx, f);
      pz = std::max(pz, z);
    }
    if (!dftx_shape_ok(*t, P->real)) continue;
    const int nr = rings_of(P->p.sampling, t->L);
    S2W_TRY(table(t->L, 1.0, &t->dftx_inv));
    S2W_TRY(table(t->L, (2.0 * kPi / (2.0 * t->L - 1.0)) * t->gscale, &t->dftx_fwd));
    ops = std::max(ops, dftx_ops_elems(*t, P->real, P->p.batch, nr));
    fx = std::max(fx, dftx_fexp_elems(P->p.batch, nr));
  }
  S2W_TRY(alloc_ws(P, (size_t)std::max<int64_t>(ops, 1), &P->dftx_ops, err));
  S2W_TRY(alloc_ws(P, (size_t)std::max<int64_t>(fx, 1), &P->dftx_fexp, err));
  if (pops > 0) {
    S2W_TRY(alloc_ws(P, (size_t)pops, &P->dftp_ops, err));
    S2W_TRY(alloc_ws(P, (size_t)pfx, &P->dftp_fexp, err));
    S2W_TRY(alloc_ws(P, (size_t)pz, &P->dftp_z, err));
  }
  return S2W_OK;
}

// Float-pair tables of one transform (offsets, allocation, the build and fold kernels).
s2w_status make_tab(s2w_plan* P, const TransformSpec& t, TabTable* tab, cudaStream_t st, std::string& err) {
  const GridTables& g = P->grids[t.grid];
  const int L = t.L, Mc = P->real ? L : 2 * L - 1, mlo = P->real ? 0 : -(L - 1);
  tab->Lp = ((g.nr + 63) / 64) * 64;
  tab->Lk = ((g.nr + 31) / 32) * 32;
  std::vector<int64_t> oi((size_t)Mc * t.nact, 0), of((size_t)Mc * t.nact, 0);
  std::vector<int> kp((size_t)Mc * t.nact, 0);
  int64_t ri = 0, rf = 0;
  for (int mi = 0; mi < Mc; ++mi)
    for (int ni = 0; ni < t.nact; ++ni) {
      const size_t idx = (size_t)mi * t.nact + ni;
      const int l0 = std::max(std::abs(mlo + mi), std::abs(t.nvals_h[ni]));
      oi[idx] = ri;
      of[idx] = rf;
      if (l0 >= L) continue;
      const int l0a = l0 & ~7, k = ((L - l0a + 31) / 32) * 32;
      kp[idx] = k;
      ri += (int64_t)k * tab->Lp;
      rf += (int64_t)tab->Lk * k;
      tab->kpmax = std::max(tab->kpmax, k);
    }
  tab->elems = std::max(ri, rf);
  S2W_TRY(upload(P, oi, &tab->off_inv, st, err));
  S2W_TRY(upload(P, of, &tab->off_fwd, st, err));
  S2W_TRY(upload(P, kp, &tab->kp, st, err));
  S2W_TRY(alloc_dev(P, (size_t)std::max<int64_t>(ri, 1), &tab->inv, err));
  S2W_TRY(alloc_dev(P, (size_t)std::max<int64_t>(rf, 1), &tab->fwd, err));
  if (tab->kpmax > 0 && launch_tab_build(g, t, *tab, Mc, mlo, st) != cudaSuccess) {
    err = "Wigner-d table kernels failed to launch";
    return S2W_ECUDA;
  }
  return S2W_OK;
}

// Float64-accurate precomputed tables (precompute = 1) for the SHT, the scaling function and
// (with_wavelets) every wavelet scale; specs with the same (L, n values) share one table.  The
// reduced modes use them for the SHT and the scaling function, which stay float64-accurate.
s2w_status build_tab_tables(s2w_plan* P, cudaStream_t st, std::string& err, bool with_wavelets) {
  std::map<std::pair<int, std::vector<int>>, TabTable*> cache;
  std::vector<TransformSpec*> specs = {&P->sht, &P->scal_t};
  if (with_wavelets)
    for (TransformSpec& t : P->wav_t) specs.push_back(&t);
  for (TransformSpec* t : specs) {
    auto key = std::make_pair(t->L, t->nvals_h);
    auto it = cache.find(key);
    if (it != cache.end()) {
      t->tab = it->second;
      continue;
    }
    TabTable* tab = new TabTable();
    P->tab_tables.push_back(tab);
    S2W_TRY(make_tab(P, *t, tab, st, err));
    cache[key] = tab;
    t->tab = tab;
  }
  return S2W_OK;
}

}  // namespace

s2w_status build_plan(const s2w_params& p, cudaStream_t st, s2w_plan* P, std::string& err) {
  if (p.L < 2 || p.L > 1024) { err = "L must satisfy 2 <= L <= 1024"; return S2W_EINVAL; }
  if (p.N < 1 || p.N > p.L) { err = "N must satisfy 1 <= N <= L"; return S2W_EINVAL; }
  if (!(p.lambda > 1.0) || !std::isfinite(p.lambda)) { err = "lambda must be > 1"; return S2W_EINVAL; }
  if (std::abs(p.spin) >= p.L) { err = "|spin| must be < L"; return S2W_EINVAL; }
  if (p.batch < 1) { err = "batch must be >= 1"; return S2W_EINVAL; }
  if (p.reality && p.spin != 0) { err = "reality requires spin 0"; return S2W_EINVAL; }
  if (p.precision != S2W_FP64 && p.precision != S2W_FP64_NATIVE && p.precision != S2W_FP32_SPLIT &&
      p.precision != S2W_BF16 && p.precision != S2W_FP64_TC) {
    err = "unknown precision mode";
    return S2W_EINVAL;
  }
  if ((p.precision == S2W_FP32_SPLIT || p.precision == S2W_BF16) && std::max(p.L, rings_of(p.sampling, p.L)) > 512) {
    err = "the reduced-precision tensor-core modes support L and the ring count <= 512 in this build";
    return S2W_EUNSUPPORTED;
  }
  if (p.precompute != 0 && p.precompute != 1) { err = "precompute must be 0 or 1"; return S2W_EINVAL; }
  if (p.sampling != S2W_SAMPLING_MW && p.sampling != S2W_SAMPLING_DH) { err = "unknown sampling"; return S2W_EINVAL; }
  if (p.sampling == S2W_SAMPLING_DH && p.L > 512) {
    err = "Driscoll-Healy sampling supports L <= 512 in this build (2L rings, one thread per ring)";
    return S2W_EUNSUPPORTED;
  }
  if (p.precision == S2W_FP64_TC && std::max(p.L, rings_of(p.sampling, p.L)) > 512) {
    err = "the sliced tensor-core contractions need L and the ring count <= 512 (exact float32 sums)";
    return S2W_EUNSUPPORTED;
  }
  if (p.precompute == 1 && p.precision == S2W_FP64_NATIVE) {
    err = "the plain float64 path computes the Wigner-d functions on the fly (precompute = 0)";
    return S2W_EUNSUPPORTED;
  }
  int J = 0;
  while (ceil_pow(p.lambda, J) < p.L) ++J;
  if (p.J0 < 0 || p.J0 > J) { err = "J0 must satisfy 0 <= J0 <= J"; return S2W_EINVAL; }

  P->p = p;
  P->native64 = p.precision == S2W_FP64_NATIVE;
  P->tensor = p.precision == S2W_FP32_SPLIT || p.precision == S2W_BF16;
  P->tcx = p.precision == S2W_FP64_TC;
  P->precompute = p.precompute == 1 && p.precision == S2W_FP64;
  P->real = p.reality != 0;
  P->Mc = P->real ? p.L : 2 * p.L - 1;
  P->mlo = P->real ? 0 : -(p.L - 1);
  P->J = J;
  P->L_phi = std::min(ceil_pow(p.lambda, p.J0), p.L);
  P->nscales = J - p.J0 + 1;
  for (int j = p.J0; j <= J; ++j) {
    int Lj = std::min(ceil_pow(p.lambda, j + 1), p.L);
    P->scale_j.push_back(j);
    P->Lj.push_back(Lj);
    P->Nj.push_back(std::min(p.N, Lj));
  }
  const int smp = p.sampling;
  P->nr = rings_of(smp, p.L);
  P->map_elems = (int64_t)P->nr * (2 * p.L - 1);
  P->scal_elems = (int64_t)rings_of(smp, P->L_phi) * (2 * P->L_phi - 1);
  P->wav_off.assign(1, 0);
  for (int s = 0; s < P->nscales; ++s)
    P->wav_off.push_back(P->wav_off.back() +
                         (int64_t)(2 * P->Nj[s] - 1) * rings_of(smp, P->Lj[s]) * (2 * P->Lj[s] - 1));
  P->wav_elems = P->wav_off.back();

  // grids for every distinct band-limit
  std::map<int, int> gidx;
  auto grid_for = [&](int L) -> int {
    auto it = gidx.find(L);
    if (it != gidx.end()) return it->second;
    int id = (int)P->grids.size();
    P->grids.emplace_back();
    gidx[L] = id;
    return id;
  };
  grid_for(p.L);
  grid_for(P->L_phi);
  for (int s = 0; s < P->nscales; ++s) grid_for(P->Lj[s]);
  for (auto& kv : gidx) S2W_TRY(build_grid(P, kv.first, st, P->grids[kv.second], err));

  Tiling tile(p.lambda);
  const int L = p.L, s = p.spin;
  // spin SHT at L: d^l_{m,-s}, multiplier (-1)^s sqrt((2l+1)/(4 pi)) (MW convention)
  {
    std::vector<cplx> mi(L), mf(L);
    for (int l = 0; l < L; ++l) {
      double v = (l >= std::abs(s)) ? ((s % 2 == 0) ? 1.0 : -1.0) * std::sqrt((2.0 * l + 1.0) / (4.0 * kPi)) : 0.0;
      mi[l] = mf[l] = v;
    }
    S2W_TRY(build_spec(P, st, P->sht, L, 1, gidx[L], {-s}, mi, mf, 1.0, err));
  }
  // scaling function at L_phi: Phi_l0 = sqrt((2l+1)/(4 pi)) sqrt(k(l / lambda^J0)); the
  // scaling map is a spin-0 function, so its harmonic multiplier is Phi_l0 (Eq. 29, Eq. 41).
  {
    const int LP = P->L_phi;
    std::vector<cplx> m(LP);
    double scale = std::pow(p.lambda, p.J0);
    for (int l = 0; l < LP; ++l)
      m[l] = (l >= std::abs(s)) ? std::sqrt((2.0 * l + 1.0) / (4.0 * kPi)) * std::sqrt(tile.k(l / scale)) : 0.0;
    S2W_TRY(build_spec(P, st, P->scal_t, LP, 1, gidx[LP], {0}, m, m, 1.0, err));
  }
  P->wav_t.resize(P->nscales);
  P->raw_t.resize(P->nscales);
  for (int sc = 0; sc < P->nscales; ++sc) {
    const int j = P->scale_j[sc], Lj = P->Lj[sc], Nj = P->Nj[sc];
    const double lj = std::pow(p.lambda, j);
    std::vector<int> act, all;
    for (int n = -(Nj - 1); n <= Nj - 1; ++n) {
      all.push_back(n);
      if (((p.N + n) % 2 + 2) % 2 == 1) act.push_back(n);
    }
    // Psi^j_ln = sqrt((2l+1)/(8 pi^2)) kappa(l / lambda^j) zeta_ln (Eq. A9)
    std::vector<cplx> mi((size_t)Lj * act.size()), mf((size_t)Lj * act.size());
    for (int l = 0; l < Lj; ++l) {
      double kap = (l >= std::abs(s)) ? tile.kappa(l / lj) : 0.0;
      for (size_t i = 0; i < act.size(); ++i) {
        cplx psi = std::sqrt((2.0 * l + 1.0) / (8.0 * kPi * kPi)) * kap * zeta(l, act[i], p.N);
        mi[(size_t)l * act.size() + i] = std::conj(psi);
        mf[(size_t)l * act.size() + i] = psi;
      }
    }
    S2W_TRY(build_spec(P, st, P->wav_t[sc], Lj, Nj, gidx[Lj], act, mi, mf, 2.0 * kPi / (2.0 * Nj - 1.0), err));
    std::vector<cplx> ri((size_t)Lj * all.size()), rf((size_t)Lj * all.size(), 1.0);
    for (int l = 0; l < Lj; ++l)
      for (size_t i = 0; i < all.size(); ++i) ri[(size_t)l * all.size() + i] = (2.0 * l + 1.0) / (8.0 * kPi * kPi);
    S2W_TRY(build_spec(P, st, P->raw_t[sc], Lj, Nj, gidx[Lj], all, ri, rf, 2.0 * kPi / (2.0 * Nj - 1.0), err));
  }

  // the reduced modes run their SHT and scaling transform on the float64-accurate sliced
  // tensor-core kernels of S2W_FP64_TC (contractions and DFTs), the wavelet scales on the
  // reduced-precision tables
  if (P->tensor) S2W_TRY(build_tc_tables(P, st, err));
  if (P->tcx || P->tensor) S2W_TRY(build_tcx_tables(P, st, err, P->tcx));
  if (P->tcx || P->tensor) S2W_TRY(build_dftx_tables(P, st, err, P->tcx));
  if (P->precompute) S2W_TRY(build_tab_tables(P, st, err, true));

  // workspaces
  const int64_t B = p.batch;
  int64_t gmax = B * (int64_t)P->nr * P->Mc;
  for (int sc = 0; sc < P->nscales; ++sc) {
    int64_t Mcj = P->real ? P->Lj[sc] : 2 * P->Lj[sc] - 1;
    gmax = std::max(gmax, B * (2 * P->Nj[sc] - 1) * (int64_t)rings_of(smp, P->Lj[sc]) * Mcj);
  }
  P->g_ws_elems = gmax;
  S2W_TRY(alloc_ws(P, (size_t)gmax, &P->g_ws, err));
  S2W_TRY(alloc_ws(P, (size_t)(B * (int64_t)L * P->Mc), &P->flm_ws, err));
  S2W_TRY(alloc_ws(P, 1, &P->err_word, err));
  if (cudaMemsetAsync(P->err_word, 0, sizeof(int), st) != cudaSuccess) { err = "memset failed"; return S2W_ECUDA; }
  if (cudaStreamSynchronize(st) != cudaSuccess) { err = "plan upload failed"; return S2W_ECUDA; }
  return S2W_OK;
}

void free_plan(s2w_plan* P) {
  for (void* q : P->owned) cudaFree(q);
  P->owned.clear();
  P->owned_bytes.clear();
  P->workspace_bytes = 0;
  for (TcTable* t : P->tc_tables) delete t;
  P->tc_tables.clear();
  for (TabTable* t : P->tab_tables) delete t;
  P->tab_tables.clear();
  for (TcxTable* t : P->tcx_tables) delete t;
  P->tcx_tables.clear();
  for (DftxTable* t : P->dftx_tables) delete t;
  P->dftx_tables.clear();
  for (DftpTable* t : P->dftp_tables) delete t;
  P->dftp_tables.clear();
}

}  // namespace s2w
