// s2w_sht_inverse_static: the inverse spin SHT with its scratch in a fixed device array.
//
// Who it is for: callers that cannot allocate device memory when they need a transform --
// for example a host application that owns every device allocation and forbids new ones
// after start-up, or code that runs while a CUDA graph is being captured (cudaMalloc is not
// allowed there) -- and that cannot borrow the plan's own workspace because another call on
// the same plan may be running on another stream.  The m-column scratch of the transform
// lives in g_static_cols, a file-scope __device__ array that every GPU which loads this
// library holds until the process exits.  Nothing here calls cudaMalloc, cudaFree or any
// allocating routine.
//
// Device address: host code cannot hand `g_static_cols` itself to a kernel (in host code that
// name is a host-side stand-in, not a device address).  Every call made while its stream is NOT
// being captured asks the runtime for the address with cudaGetSymbolAddress, with the call's
// device current, and caches it per device; a call made during stream capture uses the cached
// address without any runtime lookup, so the first call on a device must come before any
// capture.  A cached address is only valid while the device's context lives: after
// cudaDeviceReset, make one uncaptured call again before capturing.
//
// Sharing: all calls (on every plan and stream of a device) share the one array and it keeps
// the previous call's contents.  The kernels overwrite every element they later read, so
// nothing has to be cleared; two calls whose work overlaps on the GPU race on the array.
#include <mutex>
#include <string>

#include "s2w_internal.h"

namespace {

// 16 MiB: B * rings * Mc complex float64 columns, enough for 16 real MW maps at L = 256.
constexpr long long kStaticColsElems = 1 << 20;
static __device__ __align__(256) double2 g_static_cols[kStaticColsElems];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double2* g_ptr[kMaxDevices] = {};

}  // namespace

extern "C" s2w_status s2w_sht_inverse_static(const s2w_plan* cP, const void* flm, void* f, void* stream) {
  using namespace s2w;
  if (cP == nullptr) return record_error(S2W_EINVAL, "plan is NULL");
  s2w_plan* P = const_cast<s2w_plan*>(cP);
  if (flm == nullptr || f == nullptr) return record_error(S2W_EINVAL, "flm or f is NULL");
  if ((reinterpret_cast<uintptr_t>(flm) % 16) != 0 || (reinterpret_cast<uintptr_t>(f) % (P->real ? 8 : 16)) != 0)
    return record_error(S2W_EINVAL, "flm or f is misaligned");
  const long long need = (long long)P->p.batch * P->nr * P->Mc;
  if (need > kStaticColsElems)
    return record_error(S2W_EINVAL, "s2w_sht_inverse_static: batch * rings * Mc = " + std::to_string(need) +
                                        " column elements exceeds the fixed scratch of " +
                                        std::to_string(kStaticColsElems) + " (16 MiB)");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return record_error(S2W_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return record_error(S2W_EUNSUPPORTED, "device index out of range");
  cudaStream_t st = (cudaStream_t)stream;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(st, &cap);
  if (e != cudaSuccess)
    return record_error(S2W_ECUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(e));
  double2* cols = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (cap == cudaStreamCaptureStatusNone) {
      // refresh the address on every uncaptured call: it changes if the context was re-created
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_static_cols);
      if (e != cudaSuccess)
        return record_error(S2W_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_ptr[dev] = static_cast<double2*>(p);
    } else if (g_ptr[dev] == nullptr) {
      return record_error(S2W_EINVAL,
                          "s2w_sht_inverse_static: first call on this device made during stream capture; "
                          "make one call before capturing");
    }
    cols = g_ptr[dev];
  }
  P->last_stream = st;
  const TransformSpec& t = P->sht;
  const GridTables& g = P->grids[t.grid];
  CoefArgs in;
  in.coef = static_cast<const double2*>(flm);
  in.s_b = (int64_t)P->p.L * P->Mc;
  in.s_n = 0;
  in.s_l = P->Mc;
  in.mlo = P->mlo;
  ColumnArgs c;
  c.G = cols;
  c.B = P->p.batch;
  c.nact = t.nact;
  c.L = t.L;
  c.nr = P->nr;
  c.Mc = P->Mc;
  c.mlo = P->mlo;
  e = launch_wigner_inverse(P, g, t, in, c, st);
  if (e != cudaSuccess) return record_error(S2W_ECUDA, std::string("inverse contraction: ") + cudaGetErrorString(e));
  e = P->native64 ? launch_dft_inverse(P, g, t, c, f, P->map_elems, P->real, st)
                  : launch_dftc_inverse(g, t, c, f, P->map_elems, P->real, st);
  if (e != cudaSuccess) return record_error(S2W_ECUDA, std::string("azimuthal DFT (inverse): ") + cudaGetErrorString(e));
  return S2W_OK;
}
