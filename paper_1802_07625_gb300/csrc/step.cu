// Instantiation of the advection, step-control and geometry kernels.
#include <algorithm>

#include "advect.cuh"
#include "geometry.cuh"
#include "linear.cuh"
#include "outer.cuh"
#include "diagnostics.cuh"
#include "adjoint.cuh"
#include "kernels.h"

namespace cg {

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 132;
  }
  return n;
}

static inline int blocks_for(long long n, int threads, int cap) {
  long long b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (int)b;
}

// Read bandwidth probe: every thread streams 16-byte loads that bypass L1 (ld.global.cg),
// four independent loads in flight per iteration, `passes` times over the buffer; the
// sum is kept live by a store that never happens.
__global__ void __launch_bounds__(256) read_bw_kernel(const float4* __restrict__ p, long long n4, int passes,
                                                      float* sink) {
  float acc = 0.f;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (int r = 0; r < passes; ++r) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + 3 * stride < n4; i += 4 * stride) {
      const float4 a = __ldcg(p + i), b = __ldcg(p + i + stride);
      const float4 c = __ldcg(p + i + 2 * stride), d = __ldcg(p + i + 3 * stride);
      acc += (a.x + b.y) + (c.z + d.w);
    }
    for (; i < n4; i += stride) acc += __ldcg(p + i).x;
  }
  if (acc == -1.2345e-30f) sink[0] = acc;
}

void launch_read_bw(const void* p, size_t bytes, int passes, float* sink, cudaStream_t s) {
  read_bw_kernel<<<sm_count() * 8, 256, 0, s>>>((const float4*)p, (long long)(bytes / 16), passes, sink);
}

template <typename T>
void launch_heun(DevState* st, const StepParams& sp, const V2<T>* v0, const V2<T>* v1, V2<T>* d0,
                 V2<T>* d1, V2<T>* u0, V2<T>* u1, int Lx, int Ly, int mode, double h,
                 cudaGraphConditionalHandle handle, int use_cond, int blocks_per_sm, cudaStream_t s) {
  int log2Lx = 0;
  while ((1 << log2Lx) < Lx) ++log2Lx;
  // a grid-stride loop over point pairs with a few resident blocks per SM keeps the
  // number of same-address atomics of the block reductions small
  const int pairs = Lx * Ly / 2;
  if (blocks_per_sm <= 0) blocks_per_sm = 8;
  const int blocks = blocks_for(pairs, 256, sm_count() * blocks_per_sm);
  if (u0)
    launch_pdl(heun_kernel<T, true>, blocks, 256, 0, s, st, sp, v0, v1, d0, d1, u0, u1, Lx, Ly, log2Lx, mode, h,
               handle, use_cond);
  else
    launch_pdl(heun_kernel<T, false>, blocks, 256, 0, s, st, sp, v0, v1, d0, d1, (V2<T>*)nullptr,
               (V2<T>*)nullptr, Lx, Ly, log2Lx, mode, h, handle, use_cond);
}

template <typename T>
void launch_gather_u(const V2<T>* v, const V2<T>* d, V2<T>* u, int Lx, int Ly, cudaStream_t s) {
  int log2Lx = 0;
  while ((1 << log2Lx) < Lx) ++log2Lx;
  gather_u_kernel<T><<<blocks_for((long long)Lx * Ly, 256, sm_count() * 8), 256, 0, s>>>(v, d, u, Lx, Ly, log2Lx);
}

void launch_init_state(DevState* st, const StepParams& sp, cudaStream_t s) {
  init_state_kernel<<<1, 1, 0, s>>>(st, sp);
}

void launch_init_finish(DevState* st, const StepParams& sp, cudaGraphConditionalHandle handle,
                        int use_cond, cudaStream_t s) {
  init_finish_kernel<<<1, 1, 0, s>>>(st, sp, handle, use_cond);
}

template <typename T>
void launch_snapshot(const DevState* st, const V2<T>* d0, const V2<T>* d1, V2<T>* dst, int N,
                     cudaStream_t s) {
  snapshot_kernel<T><<<blocks_for(N, 256, 4096), 256, 0, s>>>(st, d0, d1, dst, N);
}

template <typename T>
void launch_map_points(const double2* in, double2* out, long long n, const V2<T>* disp, int Lx,
                       int Ly, cudaStream_t s, const int* guard) {
  if (n <= 0) return;
  map_points_kernel<T><<<blocks_for(n, 256, 1 << 16), 256, 0, s>>>(in, out, n, disp, Lx, Ly, guard);
}

void launch_raster(const double2* xy, const int* next, const int* vreg, const double* w,
                   double* acc, int Lx, int Ly, int n_vert, cudaStream_t s) {
  if (n_vert > 0)
    raster_edges_kernel<<<blocks_for(n_vert, 256, 1 << 16), 256, 0, s>>>(xy, next, vreg, w, acc, Lx,
                                                                          Ly, n_vert);
  const int t = Lx < 256 ? Lx : 256;
  row_scan_kernel<<<Ly, t, 0, s>>>(acc, Lx);
}

void launch_areas(const double2* xy, const long long* ring_off, double* sums, const int* reg_off,
                  const int* reg_rings, const double* values, int R, double* area, double* err, double* w,
                  IterInfo* info, const AreaChunks& ch, cudaStream_t s) {
  if (ch.n_chunks > 0)
    ring_chunk_kernel<<<blocks_for(ch.n_chunks * 32, 256, 1 << 20), 256, 0, s>>>(
        xy, ring_off, ch.chunk_ring, ch.ring_chunk_off, ch.n_chunks, ch.chunk_sum);
  region_area_kernel<<<blocks_for(R, 128, 1 << 16), 128, 0, s>>>(reg_off, reg_rings, ch.ring_chunk_off,
                                                                  ch.chunk_sum, R, area);
  area_sums_kernel<<<1, 1024, 0, s>>>(area, values, R, sums, info);
  region_error_kernel<<<blocks_for(R, 32, sm_count()), 32, 0, s>>>(area, values, R, sums, err, w, info);
}

void launch_collect(const DevState* st, IterInfo* info, cudaStream_t s) {
  collect_kernel<<<1, 1, 0, s>>>(st, info);
}

template <typename T>
void launch_fold_count(const V2<T>* disp, int Lx, int Ly, unsigned long long* out, cudaStream_t s) {
  cudaMemsetAsync(out, 0, sizeof(unsigned long long), s);
  cudaMemsetAsync(out + 1, 0xff, sizeof(unsigned long long), s);
  fold_kernel<T><<<blocks_for((long long)(Lx - 1) * (Ly - 1), 256, sm_count() * 4), 256, 0, s>>>(disp, Lx, Ly, out);
}

template <typename T>
void launch_phi_spectrum(const double* spec, T* phi, int Lx, int Ly, cudaStream_t s) {
  phi_spectrum_kernel<T><<<blocks_for((long long)Lx * Ly, 256, 4096), 256, 0, s>>>(spec, phi, Lx, Ly);
}

template <typename T>
void launch_linear_init(DevState* st, const StepParams& sp, const V2<T>* J, const T* rho0, V2<T>* v0, int N,
                        cudaGraphConditionalHandle handle, int use_cond, cudaStream_t s) {
  launch_pdl(linear_velocity_kernel<T>, blocks_for(N, 256, sm_count() * 8), 256, 0, s, st, J, rho0, v0,
             (V2<T>*)nullptr, N, (int)kModeInit, handle, use_cond, 0u);
  linear_init_finish_kernel<<<1, 1, 0, s>>>(st, sp, handle, use_cond);
}

template <typename T>
void launch_linear_step(DevState* st, const StepParams& sp, const V2<T>* J, const T* rho0, V2<T>* v0,
                        V2<T>* v1, V2<T>* d0, V2<T>* d1, V2<T>* u0, V2<T>* u1, int Lx, int Ly,
                        cudaGraphConditionalHandle handle, int use_cond, unsigned int max_body, int blocks_per_sm,
                        cudaStream_t s) {
  const int N = Lx * Ly;
  launch_pdl(linear_velocity_kernel<T>, blocks_for(N, 256, sm_count() * 8), 256, 0, s, st, J, rho0, v0, v1, N,
             (int)kModeLinear, handle, use_cond, max_body);
  launch_heun<T>(st, sp, v0, v1, d0, d1, u0, u1, Lx, Ly, kModeLinear, 0.0, handle, use_cond, blocks_per_sm, s);
}

void launch_blur_tables(const OuterState* o, double sigma, double* bx, double* by, int Lx, int Ly,
                        cudaStream_t s) {
  blur_tables_kernel<<<blocks_for(Lx + Ly, 256, 64), 256, 0, s>>>(o, sigma, bx, by, Lx, Ly);
}

template <typename T>
void launch_outer_commit(OuterState* o, const IterInfo* info, const V2<T>* dres, int N, cudaStream_t s) {
  outer_commit_kernel<T><<<blocks_for(N, 256, sm_count() * 4), 256, 0, s>>>(o, info, dres, N);
}

void launch_outer_decide(OuterState* o, const IterInfo* info, cudaGraphConditionalHandle handle, int after,
                         cudaStream_t s) {
  outer_decide_kernel<<<1, 1, 0, s>>>(o, info, handle, after);
}

void launch_deadline(unsigned long long* deadline, unsigned long long limit_ns, cudaStream_t s) {
  deadline_kernel<<<1, 1, 0, s>>>(deadline, limit_ns);
}

int distortion_blocks(int Lx, int Ly) { return blocks_for((long long)(Lx - 1) * (Ly - 1), 256, sm_count() * 8); }

template <typename T>
void launch_distortion(const void* const* hist, int K, int Lx, int Ly, double* part, unsigned long long* max_bits,
                       double* out, cudaStream_t s) {
  const int nb = distortion_blocks(Lx, Ly);
  cudaMemsetAsync(max_bits, 0, 2 * sizeof(unsigned long long), s);
  distortion_kernel<T><<<nb, 256, 0, s>>>(hist, K, Lx, Ly, part, max_bits);
  distortion_finish_kernel<<<1, 1, 0, s>>>(part, nb, max_bits, (Lx - 1) * (Ly - 1), out);
}

template <typename T>
void launch_inverse_points(const void* const* hist, int K, int Lx, int Ly, long long n, double2* pts,
                           cudaStream_t s) {
  if (n <= 0) return;
  inverse_points_kernel<T><<<blocks_for(n, 128, 1 << 16), 128, 0, s>>>(hist, K, Lx, Ly, n, pts);
}

int polygon_blocks(int R) { return std::max(1, std::min(R - 1, sm_count() * 4)); }

void launch_polygon_measures(const double2* xy, const double2* xy0, const long long* off, const int* reg_off,
                             const int* reg_rings, int R, double2* cent, double* alpha, double* part, double* out,
                             cudaStream_t s) {
  const int cb = blocks_for((long long)R * 32, 256, 1 << 20), ab = std::min(R, sm_count() * 4);
  const int nb = polygon_blocks(R);
  region_centroid_kernel<<<cb, 256, 0, s>>>(xy0, off, reg_off, reg_rings, R, cent);
  region_centroid_kernel<<<cb, 256, 0, s>>>(xy, off, reg_off, reg_rings, R, cent + R);
  position_error_kernel<<<nb, 256, 0, s>>>(cent, cent + R, R, part);
  aspect_ratio_kernel<<<ab, 256, 0, s>>>(xy, off, reg_off, reg_rings, R, alpha);
  polygon_finish_kernel<<<1, 1, 0, s>>>(alpha, R, part, nb, out);
  aspect_ratio_kernel<<<ab, 256, 0, s>>>(xy0, off, reg_off, reg_rings, R, alpha);
  polygon_finish_kernel<<<1, 1, 0, s>>>(alpha, R, nullptr, 0, out + 2);
}

// ---- adjoint of one outer iteration (FP64) ----------------------------------------

void launch_heun_adjoint(const double2* d, const double2* v0, const double2* v1, double h, double2* lam, double* L0,
                         double* L1, int Lx, int Ly, cudaStream_t s) {
  int log2Lx = 0;
  while ((1 << log2Lx) < Lx) ++log2Lx;
  heun_adjoint_kernel<<<blocks_for((long long)Lx * Ly, 256, sm_count() * 8), 256, 0, s>>>(d, v0, v1, h, lam, L0, L1,
                                                                                          Lx, Ly, log2Lx);
}

void launch_node_adjoint(const double* L, const double2* v, const double* rho, double* a_rho, double* a_gx,
                         double* a_gy, int Lx, int Ly, cudaStream_t s) {
  node_adjoint_kernel<<<blocks_for((long long)Lx * Ly, 256, 4096), 256, 0, s>>>(L, v, rho, a_rho, a_gx, a_gy, Lx,
                                                                               Lx * Ly);
}

void launch_spec_accumulate(const double* Crho, const double* Cx, const double* Cy, double* lam_spec, double tau,
                            int Lx, int Ly, cudaStream_t s) {
  spec_accumulate_kernel<<<std::min(Ly, sm_count() * 4), 256, 0, s>>>(Crho, Cx, Cy, lam_spec, tau, Lx, Ly);
}

void launch_spec_tail(const double* lam_spec, const double* spec, const double* bx, const double* by, double sigma,
                      double* specp, double* dsigma, int Lx, int Ly, cudaStream_t s) {
  cudaMemsetAsync(dsigma, 0, sizeof(double), s);
  spec_tail_kernel<<<blocks_for((long long)Lx * Ly, 256, 1024), 256, 0, s>>>(lam_spec, spec, bx, by, sigma, specp,
                                                                            dsigma, Lx, Ly);
}

void launch_raster_adjoint(const double2* xy, const int* next, const int* vreg, double* lam, double* grad_w,
                           int n_regions, int Lx, int Ly, int n_vert, cudaStream_t s) {
  row_suffix_kernel<<<Ly, 32, 0, s>>>(lam, Lx);
  cudaMemsetAsync(grad_w, 0, sizeof(double) * n_regions, s);
  if (n_vert > 0)
    raster_adjoint_kernel<<<blocks_for(n_vert, 256, 1 << 16), 256, 0, s>>>(xy, next, vreg, lam, grad_w, Lx, Ly,
                                                                          n_vert);
}

void launch_vertex_adjoint(const double2* xy1, const double2* xy0, const int* next, const int* prev,
                           const int* vreg, const double* dLdA, double lam, double2* g, double* lamD, int Lx,
                           int Ly, int n_vert, cudaStream_t s) {
  cudaMemsetAsync(lamD, 0, sizeof(double) * 2 * (size_t)Lx * Ly, s);
  if (n_vert <= 0) return;
  vertex_adjoint_kernel<<<blocks_for(n_vert, 256, 1 << 16), 256, 0, s>>>(xy1, xy0, next, prev, vreg, dLdA, lam, g,
                                                                        n_vert);
  map_adjoint_kernel<<<blocks_for(n_vert, 256, 1 << 16), 256, 0, s>>>(xy0, g, lamD, Lx, Ly, n_vert);
}

void launch_vertex_map_coverage(const double2* xy, const int* next, const int* vreg, const double* w,
                                const double* dens, const double2* D, const double2* lam_in, double2* lam_out,
                                int Lx, int Ly, int n_vert, cudaStream_t s) {
  if (n_vert <= 0) return;
  const int b = blocks_for(n_vert, 256, 1 << 16);
  map_jacobian_adjoint_kernel<<<b, 256, 0, s>>>(xy, D, lam_in, lam_out, Lx, Ly, n_vert);
  coverage_vertex_adjoint_kernel<<<b, 256, 0, s>>>(xy, next, vreg, w, dens, (double*)lam_out, Lx, Ly, n_vert);
}

void launch_shoelace_adjoint(const double2* xy, const int* next, const int* prev, const int* vreg,
                             const double* dLdA, double2* g, int n_vert, cudaStream_t s) {
  if (n_vert <= 0) return;
  shoelace_adjoint_kernel<<<blocks_for(n_vert, 256, 1 << 16), 256, 0, s>>>(xy, next, prev, vreg, dLdA, g, n_vert);
}

void launch_loss_vertex_adjoint(const double2* xy1, const double2* xy0, const int* next, const int* prev,
                                const int* vreg, const double* dLdA, double lam, double2* g, int n_vert,
                                cudaStream_t s) {
  if (n_vert <= 0) return;
  vertex_adjoint_kernel<<<blocks_for(n_vert, 256, 1 << 16), 256, 0, s>>>(xy1, xy0, next, prev, vreg, dLdA, lam, g,
                                                                        n_vert);
}

void launch_map_adjoint(const double2* xy_pre, const double2* g, double* lamD, int Lx, int Ly, int n_vert,
                        cudaStream_t s) {
  cudaMemsetAsync(lamD, 0, sizeof(double) * 2 * (size_t)Lx * Ly, s);
  if (n_vert <= 0) return;
  map_adjoint_kernel<<<blocks_for(n_vert, 256, 1 << 16), 256, 0, s>>>(xy_pre, g, lamD, Lx, Ly, n_vert);
}

#define CG_INSTANTIATE_STEP(T)                                                                      \
  template void launch_heun<T>(DevState*, const StepParams&, const V2<T>*, const V2<T>*, V2<T>*,    \
                               V2<T>*, V2<T>*, V2<T>*, int, int, int, double,                       \
                               cudaGraphConditionalHandle, int, int, cudaStream_t);                 \
  template void launch_gather_u<T>(const V2<T>*, const V2<T>*, V2<T>*, int, int, cudaStream_t);     \
  template void launch_snapshot<T>(const DevState*, const V2<T>*, const V2<T>*, V2<T>*, int,        \
                                   cudaStream_t);                                                   \
  template void launch_map_points<T>(const double2*, double2*, long long, const V2<T>*, int, int,   \
                                     cudaStream_t, const int*);                                     \
  template void launch_fold_count<T>(const V2<T>*, int, int, unsigned long long*, cudaStream_t);   \
  template void launch_phi_spectrum<T>(const double*, T*, int, int, cudaStream_t);                  \
  template void launch_outer_commit<T>(OuterState*, const IterInfo*, const V2<T>*, int, cudaStream_t); \
  template void launch_distortion<T>(const void* const*, int, int, int, double*, unsigned long long*,  \
                                     double*, cudaStream_t);                                        \
  template void launch_inverse_points<T>(const void* const*, int, int, int, long long, double2*,       \
                                         cudaStream_t);                                             \
  template void launch_linear_init<T>(DevState*, const StepParams&, const V2<T>*, const T*, V2<T>*, \
                                      int, cudaGraphConditionalHandle, int, cudaStream_t);          \
  template void launch_linear_step<T>(DevState*, const StepParams&, const V2<T>*, const T*, V2<T>*, \
                                      V2<T>*, V2<T>*, V2<T>*, V2<T>*, V2<T>*, int, int,             \
                                      cudaGraphConditionalHandle, int, unsigned int, int, cudaStream_t);
CG_INSTANTIATE_STEP(float)
CG_INSTANTIATE_STEP(double)

}  // namespace cg
