// The outer iteration on the device (main text: the output of one integration is the
// input of the next, repeated until the largest relative area error is below 1 %). One
// CUDA-graph launch holds a conditional WHILE node whose body rasterises, transforms,
// integrates (itself a WHILE node), stores the projected grid, maps the vertices and
// measures the areas; these kernels carry the loop's bookkeeping and decisions.
#pragma once

#include "common.cuh"

namespace cg {

// Blur factors exp(-(pi m / L)^2 sigma^2 / 2) of both axes (the Gaussian blur of the
// initial density, applied to the spectrum). sigma = o->sigma[o->iterations] inside
// the device loop (o != nullptr), else sigma_fixed.
static __global__ void blur_tables_kernel(const OuterState* o, double sigma_fixed, double* bx, double* by,
                                          int Lx, int Ly) {
  const double s = o ? o->sigma[o->iterations] : sigma_fixed;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Lx + Ly; i += gridDim.x * blockDim.x) {
    if (i < Lx) {
      const double k = kPi * i / Lx;
      bx[i] = exp(-0.5 * k * k * s * s);
    } else {
      const double k = kPi * (i - Lx) / Ly;
      by[i - Lx] = exp(-0.5 * k * k * s * s);
    }
  }
}

// After an integration: store its projected grid (the displacements in dres) in the
// next history slot, or record its failure (the vertices are then left unmapped).
template <typename T>
__global__ void outer_commit_kernel(OuterState* o, const IterInfo* info, const V2<T>* __restrict__ dres,
                                    int N) {
  if (o->status != kOuterRunning) return;
  const int ist = info->status;
  if (ist != kDone) {
    if (blockIdx.x == 0 && threadIdx.x == 0) o->status = ist == kTimeout ? kTimeout : kStepFail;
    return;
  }
  V2<T>* dst = reinterpret_cast<V2<T>*>(o->hist[o->k]);
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) dst[p] = dres[p];
}

// Before the loop (after = 0) and at the end of every iteration (after = 1): take the
// iteration's counts, then decide whether another iteration runs: not once the areas
// are within area_tol, the iteration budget is spent, an integration failed, or no
// history slot is free (the host then adds slots and launches again).
static __global__ void outer_decide_kernel(OuterState* o, const IterInfo* info, cudaGraphConditionalHandle handle,
                                           int after) {
  if (after) {
    o->accepted += info->accepted;
    o->rejected += info->rejected;
    o->t_end = info->t_end;
    o->loop_ns += info->loop_ns;
    if (o->status == kOuterRunning) {
      IterRecord* rec = reinterpret_cast<IterRecord*>(static_cast<char*>(o->hist[o->k]) + o->rec_offset);
      rec->max_err = info->max_err;
      rec->t_end = info->t_end;
      rec->blur = o->sigma[o->iterations];
      rec->accepted = info->accepted;
      rec->rejected = info->rejected;
      rec->loop_ns = info->loop_ns;
      o->k += 1;
      o->iterations += 1;
    }
  }
  o->max_err = info->max_err;
  if (o->status == kOuterRunning) {
    if (o->max_err < o->area_tol) o->status = kOuterConverged;
    else if (o->iterations >= o->max_iter) o->status = kOuterNoConverge;
    else if (o->k >= o->cap) o->status = kOuterNeedSlots;
  }
  cudaGraphSetConditional(handle, o->status == kOuterRunning ? 1u : 0u);
}

// The call's deadline: the device clock now plus the limit (0: no limit).
static __global__ void deadline_kernel(unsigned long long* deadline, unsigned long long limit_ns) {
  *deadline = limit_ns ? global_ns() + limit_ns : 0ull;
}

}  // namespace cg
