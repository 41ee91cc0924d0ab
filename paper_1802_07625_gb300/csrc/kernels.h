// Host-side launchers of the cartogram kernels (defined in spectral_*.cu, step.cu,
// geometry.cu). All launches are asynchronous on the given stream.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "common.cuh"

namespace cg {

struct LaunchCfg {
  int per_block;  // lines (rows or columns) per block
  int threads;
  size_t smem;
  int grid;
};

inline int fft_n1(int log2n) { return 1 << ((log2n + 1) / 2); }
inline int fft_stride(int log2n) {
  const int N = 1 << log2n;
  return N + N / fft_n1(log2n) + 1;  // padded signal length + one element between signals
}

// Launch shapes of the step kernels, chosen per context (heuristic defaults, or by the
// autotuner): spectral rows per block of pass 1, columns per block of pass 2 (even),
// and resident blocks per SM of the predictor-corrector kernel.
struct Tune {
  int rows = 0;
  int cols = 0;
  int heun_bps = 0;
};

inline int default_rows(int log2Lx, int Ly) {
  int S = 128 / fft_n1(log2Lx);
  if (S < 1) S = 1;
  if (S > Ly) S = Ly;
  return S;
}
inline int default_cols(int Lx, size_t esz) {
  int Wc = (esz == 4 && Lx >= 1024) ? 4 : 2;
  if (Wc > Lx) Wc = Lx;
  return Wc;
}

// pass 1 of the inverse transform: S spectral rows per block
inline LaunchCfg inv_rows_cfg(int log2Lx, int Ly, size_t esz, int S) {
  const int N = 1 << log2Lx, N1 = fft_n1(log2Lx);
  if (S <= 0) S = default_rows(log2Lx, Ly);
  LaunchCfg c;
  c.per_block = S;
  c.threads = S * N1;
  c.smem = (size_t)N * 4 * esz + (size_t)S * N * esz + (size_t)S * fft_stride(log2Lx) * 2 * esz +
           (size_t)(N + S) * esz;
  c.grid = Ly / S;
  return c;
}

// pass 2 of the inverse transform in float-float arithmetic on FP32 data (the compensated
// mixed precision): the same block shape, float-float tables and signals in shared memory
inline LaunchCfg inv_cols_ff_cfg(int log2Ly, int Lx, int Wc) {
  const int N = 1 << log2Ly, N1 = fft_n1(log2Ly);
  if (Wc <= 0) Wc = 2;
  const int S = Wc + Wc / 2;
  LaunchCfg c;
  c.per_block = Wc;
  c.threads = S * N1;
  c.smem = (size_t)N * 4 * 8 + (size_t)Wc * N * 2 * 4 + (size_t)S * fft_stride(log2Ly) * 2 * 8 + 64 * 4;
  c.grid = Lx / Wc;
  return c;
}

// pass 2 of the inverse transform: Wc columns per block
inline LaunchCfg inv_cols_cfg(int log2Ly, int Lx, size_t esz, int Wc) {
  const int N = 1 << log2Ly, N1 = fft_n1(log2Ly);
  if (Wc <= 0) Wc = default_cols(Lx, esz);
  const int S = Wc + Wc / 2;
  LaunchCfg c;
  c.per_block = Wc;
  c.threads = S * N1;
  // FP64 reads its columns and quarter-wave factors from global memory (p2_staged)
  c.smem = esz == 8 ? (size_t)N * 2 * esz + (size_t)S * fft_stride(log2Ly) * 2 * esz + 64 * esz
                    : (size_t)N * 4 * esz + (size_t)Wc * N * 2 * esz + (size_t)S * fft_stride(log2Ly) * 2 * esz +
                          64 * esz;
  c.grid = Lx / Wc;
  return c;
}

// forward transform, rows (pairs of rows per complex signal)
inline LaunchCfg fwd_rows_cfg(int log2Lx, int Ly) {
  const int N = 1 << log2Lx, N1 = fft_n1(log2Lx);
  int S = 2 * (128 / N1);
  if (S < 2) S = 2;
  if (S > Ly) S = Ly;
  LaunchCfg c;
  c.per_block = S;
  c.threads = (S / 2) * N1;
  c.smem = (size_t)N * 32 + (size_t)(S / 2) * fft_stride(log2Lx) * 16;
  c.grid = Ly / S;
  return c;
}

// forward transform, columns (pairs of columns per complex signal)
inline LaunchCfg fwd_cols_cfg(int log2Ly, int Lx) {
  const int N = 1 << log2Ly, N1 = fft_n1(log2Ly);
  int Wc = 4;
  if (Wc > Lx) Wc = Lx;
  LaunchCfg c;
  c.per_block = Wc;
  c.threads = (Wc / 2) * N1;
  c.smem = (size_t)N * 32 + (size_t)(Wc / 2) * fft_stride(log2Ly) * 16;
  c.grid = Lx / Wc;
  return c;
}

// Launch `kernel` with programmatic dependent launch allowed: it may start while the
// previous kernel on the stream drains, and waits for it (griddepcontrol.wait) before
// using its results.
template <typename... P, typename... A>
inline void launch_pdl(void (*kernel)(P...), int grid, int threads, size_t smem, cudaStream_t s,
                       A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, static_cast<P>(args)...);
}

// Pass 2 in float-float arithmetic (tables W, E: float-float pairs [N]); prepare_spectral_ff
// allows its shared memory for every column count up to 16 that fits, and reports the
// largest block it can launch.
cudaError_t prepare_spectral_ff(int log2Ly, int Lx, int* cols_max_threads);
void launch_inv_cols_ff(int log2Ly, int Lx, int Wc, const float2* AB, float2* v0, float2* v1, float* rho_out,
                        const void* W, const void* E, DevState* st, int mode, cudaStream_t s);
// The forward transform of the mixed precisions in float-float arithmetic (FP64 input and
// output; tables: float-float forward roots and quarter-wave factors [N] of each axis).
cudaError_t prepare_forward_ff(int log2Lx, int log2Ly);
void launch_fwd_ff(int log2Lx, int log2Ly, const double* rho, double* R, double* spec64, float* specT,
                   const void* Wx, const void* Ex, const void* Wy, const void* Ey, const double* bx,
                   const double* by, cudaStream_t s);

// Allow the dynamic shared memory the spectral kernels of this grid need.
template <typename T> cudaError_t prepare_spectral(int log2Lx, int log2Ly);
// Largest block size the inverse passes of this grid can launch with.
template <typename T> cudaError_t spectral_max_threads(int log2Lx, int log2Ly, int* rows_max, int* cols_max);
cudaError_t prepare_forward(int log2Lx, int log2Ly);

template <typename T>
void launch_inv_rows(int log2Lx, int Ly, int S, const T* spec, V2<T>* AB, const V2<T>* W,
                     const V2<T>* E, DevState* st, int mode, double tau,
                     cudaGraphConditionalHandle handle, int use_cond, unsigned int max_body,
                     cudaStream_t s);
template <typename T>
void launch_inv_cols(int log2Ly, int Lx, int Wc, const V2<T>* AB, V2<T>* v0, V2<T>* v1,
                     T* rho_out, const V2<T>* W, const V2<T>* E, DevState* st, int mode,
                     cudaStream_t s);
void launch_fwd_rows(int log2Lx, int log2Ly, const double* rho, double* R, const double2* Wx,
                     const double2* Ex, cudaStream_t s);
template <typename T>
void launch_fwd(int log2Lx, int log2Ly, const double* rho, double* R, double* spec64, T* specT,
                const double2* Wx, const double2* Ex, const double2* Wy, const double2* Ey,
                const double* bx, const double* by, cudaStream_t s);

// One predictor-corrector step of all grid points. u0, u1 (both null or both set): the
// cached predictor velocities by parity, read from u[p] and written to u[1 - p] (see
// heun_kernel); null: the predictor velocities are interpolated.
template <typename T>
void launch_heun(DevState* st, const StepParams& sp, const V2<T>* v0, const V2<T>* v1, V2<T>* d0,
                 V2<T>* d1, V2<T>* u0, V2<T>* u1, int Lx, int Ly, int mode, double h,
                 cudaGraphConditionalHandle handle, int use_cond, int blocks_per_sm, cudaStream_t s);
// u = v interpolated at the grid points displaced by d (the cached predictor velocities
// at the start of an integration).
template <typename T>
void launch_gather_u(const V2<T>* v, const V2<T>* d, V2<T>* u, int Lx, int Ly, cudaStream_t s);
int sm_count();
// Read `bytes` (a multiple of 16) of p, `passes` times, bypassing L1.
void launch_read_bw(const void* p, size_t bytes, int passes, float* sink, cudaStream_t s);

// persistent integration kernel (persist.cu)
constexpr int kIntegrateThreads = 256;
template <typename T> cudaError_t prepare_integrate(size_t smem, int* blocks_per_sm);
template <typename T>
cudaError_t launch_integrate(const IntegrateArgs<T>& a, int grid, size_t smem, cudaStream_t s);
void launch_init_state(DevState* st, const StepParams& sp, cudaStream_t s);
void launch_init_finish(DevState* st, const StepParams& sp, cudaGraphConditionalHandle handle,
                        int use_cond, cudaStream_t s);
template <typename T>
void launch_snapshot(const DevState* st, const V2<T>* d0, const V2<T>* d1, V2<T>* dst, int N,
                     cudaStream_t s);
template <typename T>
void launch_phi_spectrum(const double* spec, T* phi, int Lx, int Ly, cudaStream_t s);
// Linear-equalisation flow: the velocity at t = 0 at the grid points (into v0) and the
// first step; one attempted step (the velocity at its end, then the predictor-corrector
// step of all points with the linear flow's controller).
template <typename T>
void launch_linear_init(DevState* st, const StepParams& sp, const V2<T>* J, const T* rho0, V2<T>* v0, int N,
                        cudaGraphConditionalHandle handle, int use_cond, cudaStream_t s);
template <typename T>
void launch_linear_step(DevState* st, const StepParams& sp, const V2<T>* J, const T* rho0, V2<T>* v0,
                        V2<T>* v1, V2<T>* d0, V2<T>* d1, V2<T>* u0, V2<T>* u1, int Lx, int Ly,
                        cudaGraphConditionalHandle handle, int use_cond, unsigned int max_body, int blocks_per_sm,
                        cudaStream_t s);
// Outer iteration on the device: blur factors (of o->sigma[o->iterations], or of sigma
// when o is null), storing an integration's projected grid, and the loop decision.
void launch_blur_tables(const OuterState* o, double sigma, double* bx, double* by, int Lx, int Ly,
                        cudaStream_t s);
template <typename T>
void launch_outer_commit(OuterState* o, const IterInfo* info, const V2<T>* dres, int N, cudaStream_t s);
void launch_outer_decide(OuterState* o, const IterInfo* info, cudaGraphConditionalHandle handle, int after,
                         cudaStream_t s);
// *deadline = device clock + limit_ns (0: no deadline), at the start of a call.
void launch_deadline(unsigned long long* deadline, unsigned long long limit_ns, cudaStream_t s);
// Polygon-level measures (SI section 4) of the map with vertices xy against the input map
// xy0: out[0] mean aspect ratio of xy's regions, out[1] relative position error, out[2] mean
// aspect ratio of xy0's regions. Scratch: cent [2R], alpha [R], part [polygon_blocks(R)].
int polygon_blocks(int R);
void launch_polygon_measures(const double2* xy, const double2* xy0, const long long* off, const int* reg_off,
                             const int* reg_rings, int R, double2* cent, double* alpha, double* part, double* out,
                             cudaStream_t s);
// Diagnostics of the composed projection (history grids hist[0..K)): angular
// distortion into out[4] (part: 2 * distortion_blocks doubles, max_bits: 2 words), and
// the preimages of n points, in place.
int distortion_blocks(int Lx, int Ly);
template <typename T>
void launch_distortion(const void* const* hist, int K, int Lx, int Ly, double* part, unsigned long long* max_bits,
                       double* out, cudaStream_t s);
template <typename T>
void launch_inverse_points(const void* const* hist, int K, int Lx, int Ly, long long n, double2* pts,
                           cudaStream_t s);
// Adjoint of one outer iteration (FP64): one predictor-corrector step backwards
// (positions d before the step, fields v0, v1; lam in place; field adjoints scattered
// into L0, L1 [N][2]); a level's field adjoint through v = -g/rho; its transposed
// transforms accumulated into the spectrum adjoint; the blur derivative and the input of
// the density adjoint; the rasteriser's adjoint (lam: density adjoint, overwritten by its
// row suffix sums); the loss adjoint of the mapped vertices scattered into the final
// displacements' adjoint lamD [N][2].
void launch_heun_adjoint(const double2* d, const double2* v0, const double2* v1, double h, double2* lam, double* L0,
                         double* L1, int Lx, int Ly, cudaStream_t s);
void launch_node_adjoint(const double* L, const double2* v, const double* rho, double* a_rho, double* a_gx,
                         double* a_gy, int Lx, int Ly, cudaStream_t s);
void launch_spec_accumulate(const double* Crho, const double* Cx, const double* Cy, double* lam_spec, double tau,
                            int Lx, int Ly, cudaStream_t s);
void launch_spec_tail(const double* lam_spec, const double* spec, const double* bx, const double* by, double sigma,
                      double* specp, double* dsigma, int Lx, int Ly, cudaStream_t s);
void launch_raster_adjoint(const double2* xy, const int* next, const int* vreg, double* lam, double* grad_w,
                           int n_regions, int Lx, int Ly, int n_vert, cudaStream_t s);
void launch_vertex_adjoint(const double2* xy1, const double2* xy0, const int* next, const int* prev,
                           const int* vreg, const double* dLdA, double lam, double2* g, double* lamD, int Lx,
                           int Ly, int n_vert, cudaStream_t s);
// Vertex adjoints through several outer iterations: the input vertices X_k of iteration k
// through the map X_{k+1} = X_k + D_k(X_k) (lam_in: adjoint of X_{k+1}) and the exact
// coverage of the rasteriser (dens: density adjoint per cell, w: the iteration's region
// weights) into lam_out; the region areas' adjoint dLdA added through the shoelace sums;
// the loss's vertex adjoint (areas of xy1 and the displacement penalty from xy0); the
// final displacements' adjoint of a map from xy_pre (lamD [N][2], zeroed first).
void launch_vertex_map_coverage(const double2* xy, const int* next, const int* vreg, const double* w,
                                const double* dens, const double2* D, const double2* lam_in, double2* lam_out,
                                int Lx, int Ly, int n_vert, cudaStream_t s);
void launch_shoelace_adjoint(const double2* xy, const int* next, const int* prev, const int* vreg,
                             const double* dLdA, double2* g, int n_vert, cudaStream_t s);
void launch_loss_vertex_adjoint(const double2* xy1, const double2* xy0, const int* next, const int* prev,
                                const int* vreg, const double* dLdA, double lam, double2* g, int n_vert,
                                cudaStream_t s);
void launch_map_adjoint(const double2* xy_pre, const double2* g, double* lamD, int Lx, int Ly, int n_vert,
                        cudaStream_t s);
template <typename T>
void launch_fold_count(const V2<T>* disp, int Lx, int Ly, unsigned long long* out, cudaStream_t s);
template <typename T>
void launch_map_points(const double2* in, double2* out, long long n, const V2<T>* disp, int Lx,
                       int Ly, cudaStream_t s, const int* guard = nullptr);

void launch_raster(const double2* xy, const int* next, const int* vreg, const double* w,
                   double* acc, int Lx, int Ly, int n_vert, cudaStream_t s);
// Region areas, sums[0..1] = (sum A, sum V) (scratch of two doubles), relative errors,
// rasterisation weights and the largest |error| into info->max_err.
void launch_areas(const double2* xy, const long long* ring_off, double* sums, const int* reg_off,
                  const int* reg_rings, const double* values, int R, double* area, double* err, double* w,
                  IterInfo* info, const AreaChunks& ch, cudaStream_t s);
void launch_collect(const DevState* st, IterInfo* info, cudaStream_t s);

}  // namespace cg
