// aim_matvec_noalloc: the operator product of aim_matvec with its grid work space taken
// from a fixed device array instead of the context's allocations.
//
// Who needs it: callers that may not allocate device memory once they are running --
// a real-time or certified code path that fixes its memory budget at start-up, a host
// application whose device memory belongs to another allocator (a framework's caching
// pool that must not be bypassed), or a process running under a hard device-memory
// quota.  The entry point allocates nothing: no cudaMalloc, no cudaFree, no allocating
// library call.
//
// The work space is one file-scope __device__ array of kNoAllocScratchBytes (16 MiB),
// which every GPU that loads this library holds until the process exits.  Host code
// cannot pass the array's name to a kernel (in host code it is a host-side stand-in, not
// a device address), so the device address is looked up with cudaGetSymbolAddress once
// per device, by the first call made on that device, with the device current (guarded by
// a per-device once-flag, so concurrent first calls from several host threads are safe).
// The cached address does not survive cudaDeviceReset: a process that resets a device
// must not call this entry point on that device afterwards.
#include <cstring>
#include <mutex>

#include "aim_internal.h"
#include "operator.h"

namespace {

constexpr size_t kNoAllocScratchBytes = 16u << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

void* g_scratch_addr[kMaxDevices] = {nullptr};
std::once_flag g_scratch_once[kMaxDevices];

size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// swaps the context's grid work buffers for the fixed array and back
struct ScratchSwap {
  aim_ctx* c;
  void *A, *Bf, *P;
  bool prof;
  ScratchSwap(aim_ctx* c_, char* base, size_t a, size_t bf) : c(c_), A(c_->d_A), Bf(c_->d_Bf), P(c_->d_P) {
    c->d_A = base;
    c->d_Bf = base + a;
    c->d_P = base + a + bf;
    prof = c->prof.on;
    c->prof.on = false;  // event timing would create events: not on this path
  }
  ~ScratchSwap() {
    c->d_A = A;
    c->d_Bf = Bf;
    c->d_P = P;
    c->prof.on = prof;
  }
};

}  // namespace

extern "C" int aim_matvec_noalloc(aim_ctx* c, int32_t m, int32_t nb, const aim_c128* x, aim_c128* y) {
  if (!c) return AIM_ERR_ARG;
  try {
    if (!x || !y || nb < 1 || nb > c->batch_max || m < 0 || m > c->n_delays)
      throw AimError{AIM_ERR_ARG, "aim_matvec_noalloc: bad delay, batch or pointer"};
    const size_t es = c->precision == AIM_C64 ? sizeof(float2) : sizeof(double2);
    const size_t a = round256(grid_a_elems(c, nb) * es);
    const size_t bf = round256(grid_bf_elems(c, nb) * es);
    const size_t p = round256(grid_p_elems(c, nb) * es);
    if (a + bf + p > kNoAllocScratchBytes)
      throw AimError{AIM_ERR_ARG, "aim_matvec_noalloc: grid work space of " + std::to_string(a + bf + p) +
                                      " bytes exceeds the fixed 16 MiB array (use aim_matvec)"};
    int dev = 0;
    AIM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) throw AimError{AIM_ERR_ARG, "aim_matvec_noalloc: device index"};
    // set-up, once per device with that device current (a failure leaves the flag unset,
    // so a later call retries)
    std::call_once(g_scratch_once[dev], [] {
      void* ptr = nullptr;
      AIM_CUDA(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
      int d = 0;
      AIM_CUDA(cudaGetDevice(&d));
      g_scratch_addr[d] = ptr;
    });
    const size_t n = (size_t)nb * c->ns;
    const double2* xs = reinterpret_cast<const double2*>(x);
    if (!is_device_ptr(x)) {
      AIM_CUDA(cudaMemcpyAsync(c->d_x, x, n * sizeof(double2), cudaMemcpyHostToDevice, c->stream));
      xs = c->d_x;
    }
    const bool ydev = is_device_ptr(y);
    double2* ys = ydev ? reinterpret_cast<double2*>(y) : c->d_y;
    {
      ScratchSwap sw(c, static_cast<char*>(g_scratch_addr[dev]), a, bf);
      op_apply(c, m, nb, xs, nullptr, nullptr, 1.0, nullptr, ys);
    }
    if (!ydev) AIM_CUDA(cudaMemcpyAsync(y, ys, n * sizeof(double2), cudaMemcpyDeviceToHost, c->stream));
    AIM_CUDA(cudaStreamSynchronize(c->stream));
    return AIM_OK;
  } catch (const AimError& e) {
    c->err = e.msg;
    return e.code;
  } catch (...) {
    c->err = "aim_matvec_noalloc: unexpected exception";
    return AIM_ERR_ARG;
  }
}
