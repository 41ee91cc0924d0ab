// Velocity field from a caller's spectrum without any device allocation.
//
// Some callers cannot allocate GPU memory at the time they need the field: a host
// application that hands this library a fixed device-memory budget and owns every
// allocation itself, or a real-time loop that must not call the allocator because
// cudaMalloc and cudaFree may synchronise the device and take unbounded time. This
// entry point keeps its scratch (the transposed intermediate of the two transform
// passes, the transform tables and the reduction state) in one file-scope device array
// of fixed size; the caller passes the input spectrum and the output field. The array
// is created when the library is loaded onto a GPU and held by every GPU that loads the
// library until the process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <stdint.h>

#include "../../include/cartogram.h"
#include "kernels.h"

namespace {

constexpr int kMaxCells = 512 * 512;  // largest Lx * Ly accepted
constexpr size_t kABBytes = (size_t)kMaxCells * sizeof(float2);
constexpr size_t kTableBytes = 4 * 512 * sizeof(float2);
constexpr size_t kStateBytes = (sizeof(cg::DevState) + 255) / 256 * 256;
constexpr size_t kScratchBytes = kABBytes + kTableBytes + kStateBytes;

// Shared scratch of every call on a device; holds the last call's contents.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Per-device set-up, with that device current: the device address of the scratch array
// (the host-side name of the array is not a device address) and the shared-memory limits
// of the transform kernels for every accepted size.
int setup_device(int dev, void** ptr) {
  std::lock_guard<std::mutex> lock(g_mutex);
  if (dev < 0 || dev >= kMaxDevices) return CG_EINVAL;
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return CG_ECUDA;
    }
    for (int lx = 3; lx <= 9; ++lx)
      for (int ly = 3; ly <= 9; ++ly)
        if ((1 << (lx + ly)) <= kMaxCells && cg::prepare_spectral<float>(lx, ly) != cudaSuccess) {
          cudaGetLastError();
          return CG_ECUDA;
        }
    g_scratch_ptr[dev] = p;
  }
  *ptr = g_scratch_ptr[dev];
  return CG_OK;
}

// Inter-step twiddles of the four-step FFT ([k2][n1] order) and quarter-wave factors of a
// length-N axis, in FP32.
__global__ void noalloc_tables_kernel(float2* W, float2* E, int N, int N1) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) {
    const int n1 = p % N1, k2 = p / N1;
    double s, c;
    sincospi(2.0 * (double)((n1 * k2) % N) / N, &s, &c);
    W[p] = make_float2((float)c, (float)s);
    sincospi((double)p / (2.0 * N), &s, &c);
    E[p] = make_float2((float)c, (float)s);
  }
}

bool pow2_between(int n, int lo, int hi) { return n >= lo && n <= hi && (n & (n - 1)) == 0; }

int log2i(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

// Device (or managed) memory of device `dev`.
bool is_device_memory(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

}  // namespace

extern "C" int cartogram_velocity_noalloc(int Lx, int Ly, const float* spec, double t, float* v_out,
                                          void* stream) {
  if (!pow2_between(Lx, 8, 512) || !pow2_between(Ly, 8, 512) || Lx * Ly > kMaxCells) return CG_EINVAL;
  if (!spec || !v_out || !(t >= 0.0) || t > 1e300) return CG_EINVAL;
  // the transform passes read the spectrum and write the field with 16-byte vector accesses
  if (((uintptr_t)spec & 15) || ((uintptr_t)v_out & 15)) return CG_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CG_ECUDA;
  if (!is_device_memory(spec, dev) || !is_device_memory(v_out, dev)) return CG_EINVAL;
  void* base = nullptr;
  const int r = setup_device(dev, &base);
  if (r != CG_OK) return r;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* b = (unsigned char*)base;
  float2* ABt = (float2*)b;
  float2* Wx = (float2*)(b + kABBytes);
  float2* Ex = Wx + 512;
  float2* Wy = Ex + 512;
  float2* Ey = Wy + 512;
  cg::DevState* st = (cg::DevState*)(b + kABBytes + kTableBytes);
  const int log2Lx = log2i(Lx), log2Ly = log2i(Ly);
  // the reduction state must start at zero; everything else is overwritten
  if (cudaMemsetAsync(st, 0, sizeof(cg::DevState), s) != cudaSuccess) return CG_ECUDA;
  // The tables kernels stay plain launches (no programmatic dependent launch) placed
  // before the row pass: that pass starts its bulk copies of the tables before it waits
  // on its predecessor, which is safe only because a full kernel boundary separates it
  // from the kernels that write them.
  noalloc_tables_kernel<<<(Lx + 255) / 256, 256, 0, s>>>(Wx, Ex, Lx, cg::fft_n1(log2Lx));
  noalloc_tables_kernel<<<(Ly + 255) / 256, 256, 0, s>>>(Wy, Ey, Ly, cg::fft_n1(log2Ly));
  cg::launch_inv_rows<float>(log2Lx, Ly, cg::default_rows(log2Lx, Ly), spec, ABt, Wx, Ex, st, cg::kModeFixed,
                             t, 0, 0, 0u, s);
  cg::launch_inv_cols<float>(log2Ly, Lx, cg::default_cols(Lx, sizeof(float)), ABt, (float2*)v_out, nullptr,
                             nullptr, Wy, Ey, st, cg::kModeFixed, s);
  if (cudaGetLastError() != cudaSuccess) return CG_ECUDA;
  return CG_OK;
}
