// Runtime around the transforms: an autotuner for the launch shapes of a plan and a batch
// executor that runs the transforms of several plans (maps of mixed band-limit and spin) as
// one CUDA graph.
//
// Autotuner: for every transform of the plan (spin SHT, scaling function, each wavelet scale)
// it times the candidate thread counts of the DFT kernels and the candidate maps-per-block of
// the on-the-fly inverse contraction on the plan's own workspace and shapes, and keeps the
// fastest.  Batch: the plans' calls are captured once on a fork of streams (one per plan, so
// independent transforms overlap on the GPU) into a graph that one cudaGraphLaunch replays; the
// I/O buffers are fixed at creation.
#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "s2w_internal.h"

using namespace s2w;

namespace {

struct Timer {
  cudaEvent_t a = nullptr, b = nullptr;
  Timer() {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
  }
  ~Timer() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
};

// median-free: best of `reps` timings of fn() on st, in ms (infinity on a launch error)
template <class F>
float time_best(cudaStream_t st, Timer& tm, int reps, F fn) {
  float best = 1e30f;
  if (fn() != cudaSuccess) return best;   // warm-up
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(tm.a, st);
    if (fn() != cudaSuccess) return 1e30f;
    cudaEventRecord(tm.b, st);
    if (cudaEventSynchronize(tm.b) != cudaSuccess) return 1e30f;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, tm.a, tm.b);
    best = std::min(best, ms);
  }
  return best;
}

}  // namespace

struct s2w_batch {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;
  std::vector<s2w_plan*> plans;
};

extern "C" {

s2w_status s2w_plan_autotune(s2w_plan* P, void* stream) {
  if (P == nullptr) return record_error(S2W_EINVAL, "plan is NULL");
  if (P->native64) return S2W_OK;   // the plain float64 path has no tunable shapes
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<TransformSpec*> specs = {&P->sht, &P->scal_t};
  for (TransformSpec& t : P->wav_t) specs.push_back(&t);
  // pixel scratch for the largest transform (zeroed; the timing does not depend on the values)
  int64_t pix = 0;
  for (TransformSpec* t : specs)
    pix = std::max<int64_t>(pix, (int64_t)(2 * t->N - 1) * rings_of(P->p.sampling, t->L) * (2 * t->L - 1));
  void* buf = nullptr;
  const size_t eb = P->real ? sizeof(double) : sizeof(double2);
  if (cudaMalloc(&buf, (size_t)P->p.batch * pix * eb) != cudaSuccess) {
    cudaGetLastError();
    return record_error(S2W_ENOMEM, "autotune scratch allocation failed");
  }
  if (cudaMemsetAsync(buf, 0, (size_t)P->p.batch * pix * eb, st) != cudaSuccess ||
      cudaMemsetAsync(P->g_ws, 0, (size_t)P->g_ws_elems * sizeof(double2), st) != cudaSuccess ||
      cudaMemsetAsync(P->flm_ws, 0, (size_t)P->p.batch * P->p.L * P->Mc * sizeof(double2), st) != cudaSuccess) {
    cudaFree(buf);
    return record_error(S2W_ECUDA, "autotune scratch initialisation failed");
  }
  Timer tm;
  const int cand_threads[] = {128, 256, 384, 512};
  const int cand_mb[] = {4, 8, 16};
  for (TransformSpec* t : specs) {
    const GridTables& g = P->grids[t->grid];
    ColumnArgs c;
    c.G = P->g_ws;
    c.B = P->p.batch;
    c.nact = t->nact;
    c.L = t->L;
    c.nr = g.nr;
    c.Mc = P->real ? t->L : 2 * t->L - 1;
    c.mlo = P->real ? 0 : -(t->L - 1);
    const int64_t pix_sb = (int64_t)(2 * t->N - 1) * g.nr * (2 * t->L - 1);
    // S2W_FP64_TC: every DFT form with tables for the transform is timed, each with every thread
    // count (the block size of the per-ring kernels: the prime-factor form's prologues and
    // synthesis, the direct form's prologues, the compensated kernels)
    for (int dir = 0; dir < 2; ++dir) {
      const bool fwd = dir == 0;
      int& form = fwd ? t->dft_form_fwd : t->dft_form_inv;
      int& threads = fwd ? t->dft_threads_fwd : t->dft_threads_inv;
      // sliced transforms: S2W_FP64_TC's, and the reduced modes' SHT and scaling transform
      const bool sliced = P->tcx || t->tcx != nullptr;
      std::vector<int> forms = {kDftComp};
      if (sliced && (fwd ? (const void*)t->dftx_fwd : (const void*)t->dftx_inv) != nullptr) forms.push_back(kDftGemm);
      if (sliced && !P->slice_diag7 && (fwd ? (const void*)t->dftp_fwd : (const void*)t->dftp_inv) != nullptr)
        forms.push_back(kDftPfa);
      if (!sliced) forms = {kDftAuto};
      float best = 1e30f;
      int pick_th = threads, pick_form = form;
      for (int fm : forms)
        for (int th : cand_threads) {
          threads = th;
          form = fm;
          const float ms = time_best(st, tm, 3, [&] {
            return fwd ? launch_dft_forward_mode(P, g, *t, buf, pix_sb, c, st)
                       : launch_dft_inverse_mode(P, g, *t, c, buf, pix_sb, st);
          });
          if (ms < best) best = ms, pick_th = th, pick_form = fm;
        }
      threads = pick_th;
      form = pick_form;
    }
    float best = 1e30f;
    int pick = 0;
    if (t->tc == nullptr && t->tab == nullptr && t->tcx == nullptr) {
      CoefArgs in;
      in.coef = P->flm_ws;
      in.s_b = (int64_t)P->p.L * P->Mc;
      in.s_n = 0;
      in.s_l = P->Mc;
      in.mlo = P->mlo;
      best = 1e30f;
      pick = t->inv_mb;
      for (int mb : cand_mb) {
        t->inv_mb = mb;
        const float ms = time_best(st, tm, 3, [&] { return launch_wigner_inverse(P, g, *t, in, c, st); });
        if (ms < best) best = ms, pick = mb;
      }
      t->inv_mb = pick;
    }
  }
  cudaError_t e = cudaStreamSynchronize(st);
  cudaFree(buf);
  if (e != cudaSuccess) return record_error(S2W_ECUDA, std::string("autotune: ") + cudaGetErrorString(e));
  // the timed launches wrote garbage into the workspaces only; no output buffer was touched
  return S2W_OK;
}

s2w_status s2w_plan_launch_shapes(const s2w_plan* P, int transform, int* dft_threads_fwd, int* dft_threads_inv,
                                  int* inv_mb) {
  if (P == nullptr) return record_error(S2W_EINVAL, "plan is NULL");
  if (transform < 0 || transform > P->nscales + 1) return record_error(S2W_EINVAL, "transform index out of range");
  const TransformSpec& t = transform == 0 ? P->sht : transform == 1 ? P->scal_t : P->wav_t[transform - 2];
  if (dft_threads_fwd) *dft_threads_fwd = t.dft_threads_fwd;
  if (dft_threads_inv) *dft_threads_inv = t.dft_threads_inv;
  if (inv_mb) *inv_mb = t.inv_mb;
  return S2W_OK;
}

s2w_status s2w_plan_set_dft_forms(s2w_plan* P, int transform, int fwd, int inv) {
  if (P == nullptr) return record_error(S2W_EINVAL, "plan is NULL");
  if (transform < 0 || transform > P->nscales + 1) return record_error(S2W_EINVAL, "transform index out of range");
  if (fwd < -1 || fwd > 2 || inv < -1 || inv > 2) return record_error(S2W_EINVAL, "DFT form must be -1, 0, 1 or 2");
  TransformSpec& t = transform == 0 ? P->sht : transform == 1 ? P->scal_t : P->wav_t[transform - 2];
  auto to_form = [&](int code, bool f) -> int {
    if (code < 0) return kDftAuto;
    if (code == 0) return kDftComp;
    const void* tab = code == 2 ? (f ? (const void*)t.dftp_fwd : (const void*)t.dftp_inv)
                                : (f ? (const void*)t.dftx_fwd : (const void*)t.dftx_inv);
    if (code == 2 && P->slice_diag7) return -1;   // the prime-factor kernel sums diagonals 0..6 only
    return ((P->tcx || t.tcx != nullptr) && tab != nullptr) ? (code == 2 ? kDftPfa : kDftGemm) : -1;
  };
  const int ff = to_form(fwd, true), fi = to_form(inv, false);
  if (ff < 0 || fi < 0)
    return record_error(S2W_EUNSUPPORTED, "that DFT form has no tables for this transform (S2W_FP64_TC, and the SHT and scaling transform of the reduced modes)");
  t.dft_form_fwd = ff;
  t.dft_form_inv = fi;
  return S2W_OK;
}

s2w_status s2w_plan_dft_forms(const s2w_plan* P, int transform, int* tc_fwd, int* tc_inv) {
  if (P == nullptr) return record_error(S2W_EINVAL, "plan is NULL");
  if (transform < 0 || transform > P->nscales + 1) return record_error(S2W_EINVAL, "transform index out of range");
  const TransformSpec& t = transform == 0 ? P->sht : transform == 1 ? P->scal_t : P->wav_t[transform - 2];
  auto code = [&](bool fwd) {
    const int f = dft_form_used(P, t, fwd);
    return f == kDftPfa ? 2 : f == kDftGemm ? 1 : 0;
  };
  if (tc_fwd) *tc_fwd = code(true);
  if (tc_inv) *tc_inv = code(false);
  return S2W_OK;
}

s2w_status s2w_batch_create(s2w_plan* const* plans, int count, const void* const* in, void* const* wav,
                            void* const* scal, void* const* out, int what, void* stream, s2w_batch** res) {
  if (res == nullptr) return record_error(S2W_EINVAL, "out is NULL");
  *res = nullptr;
  if (plans == nullptr || count < 1) return record_error(S2W_EINVAL, "no plans");
  if (what < 0 || what > 2) return record_error(S2W_EINVAL, "what must be 0 (analysis), 1 (synthesis) or 2 (both)");
  for (int i = 0; i < count; ++i) {
    if (plans[i] == nullptr) return record_error(S2W_EINVAL, "a plan is NULL");
    for (int k = 0; k < i; ++k)
      if (plans[k] == plans[i]) return record_error(S2W_EINVAL, "a plan appears twice (its workspace would be shared)");
  }
  s2w_batch* Bt = new (std::nothrow) s2w_batch();
  if (Bt == nullptr) return record_error(S2W_ENOMEM, "host allocation failed");
  auto fail = [&](s2w_status s, const std::string& m) {
    for (cudaEvent_t e : Bt->events) cudaEventDestroy(e);
    for (cudaStream_t q : Bt->streams) cudaStreamDestroy(q);
    if (Bt->exec) cudaGraphExecDestroy(Bt->exec);
    if (Bt->graph) cudaGraphDestroy(Bt->graph);
    delete Bt;
    return record_error(s, m);
  };
  cudaStream_t origin = nullptr;
  if (cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking) != cudaSuccess) return fail(S2W_ECUDA, "stream");
  Bt->streams.push_back(origin);
  for (int i = 0; i <= count; ++i) {
    cudaEvent_t e;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return fail(S2W_ECUDA, "event");
    Bt->events.push_back(e);
  }
  for (int i = 0; i < count; ++i) {
    cudaStream_t q;
    if (cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking) != cudaSuccess) return fail(S2W_ECUDA, "stream");
    Bt->streams.push_back(q);
    Bt->plans.push_back(plans[i]);
  }
  if (cudaStreamBeginCapture(origin, cudaStreamCaptureModeRelaxed) != cudaSuccess)
    return fail(S2W_ECUDA, "stream capture could not begin");
  cudaEventRecord(Bt->events[count], origin);
  s2w_status s = S2W_OK;
  for (int i = 0; i < count && s == S2W_OK; ++i) {
    s2w_plan* P = plans[i];
    cudaStream_t q = Bt->streams[i + 1];
    cudaStreamWaitEvent(q, Bt->events[count], 0);
    const bool tr = P->trace_on;
    P->trace_on = false;   // no tracer events inside the graph
    if (what != 1) s = s2w_forward(P, in ? in[i] : nullptr, wav[i], scal[i], q);
    if (s == S2W_OK && what != 0) s = s2w_inverse(P, wav[i], scal[i], out[i], q);
    P->trace_on = tr;
    cudaEventRecord(Bt->events[i], q);
    cudaStreamWaitEvent(origin, Bt->events[i], 0);
  }
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(origin, &graph);
  Bt->graph = graph;
  if (s != S2W_OK) return fail(s, std::string("capture: ") + s2w_last_error());
  if (ec != cudaSuccess || graph == nullptr) return fail(S2W_ECUDA, std::string("capture: ") + cudaGetErrorString(ec));
  if (cudaGraphInstantiate(&Bt->exec, graph, 0) != cudaSuccess) return fail(S2W_ECUDA, "graph instantiation failed");
  (void)stream;
  *res = Bt;
  return S2W_OK;
}

s2w_status s2w_batch_launch(s2w_batch* Bt, void* stream) {
  if (Bt == nullptr) return record_error(S2W_EINVAL, "batch is NULL");
  const cudaError_t e = cudaGraphLaunch(Bt->exec, (cudaStream_t)stream);
  if (e != cudaSuccess) return record_error(S2W_ECUDA, std::string("graph launch: ") + cudaGetErrorString(e));
  for (s2w_plan* P : Bt->plans) P->last_stream = (cudaStream_t)stream;
  return S2W_OK;
}

s2w_status s2w_batch_destroy(s2w_batch* Bt) {
  if (Bt == nullptr) return record_error(S2W_EINVAL, "batch is NULL");
  if (Bt->exec) cudaGraphExecDestroy(Bt->exec);
  if (Bt->graph) cudaGraphDestroy(Bt->graph);
  for (cudaEvent_t e : Bt->events) cudaEventDestroy(e);
  for (cudaStream_t q : Bt->streams) cudaStreamDestroy(q);
  delete Bt;
  return S2W_OK;
}

}  // extern "C"
