// Geometry kernels: exact-coverage rasterisation of the regions, ring and region
// areas with the relative area errors, and mapping points through a projected grid.
#pragma once

#include "common.cuh"

namespace cg {

// ---------------------------------------------------------------------------
// Rasterisation: rho'[j][i] = sum_regions w_r * area(region_r intersect cell_ij),
// w_r = (V_r / A_r) / (sum V / sum A) - 1 (the density relative to the map mean,
// minus one; the margin of the box, covered by no region, gets 0).
//
// A ring's coverage of cell (i, j) is sum over its edges of -dy * clamp(i+1 - x(y), 0, 1)
// integrated along the edge (the winding number of a leftward ray). Every edge is cut
// at the grid lines into pieces inside one cell; a piece in cell (i, j) with vertical
// extent dy and mean abscissa x_m adds -w dy (i+1 - x_m) to D[j][i] and -w dy (x_m - i)
// to D[j][i+1]; the prefix sum of D along each row is the coverage-weighted density.
// ---------------------------------------------------------------------------
// Deposit of one piece inside cell (i, j): c = -w dy to D[j][i] and D[j][i+1] in the
// proportions (i+1 - x_m) and (x_m - i); a piece left of the box (i < 0) deposits all of
// c in column 0.
__device__ __forceinline__ void raster_piece(double ax, double bx, double pdy, int i, int j, double wt,
                                             double* __restrict__ acc, int Lx, int Ly) {
  if (pdy == 0.0 || j < 0 || j >= Ly) return;
  const double c = -wt * pdy;
  double* row = acc + (size_t)j * Lx;
  if (i < 0) {
    atomicAdd(row, c);
  } else if (i < Lx) {
    const double t = c * (0.5 * (ax + bx) - (double)i);
    atomicAdd(row + i, c - t);
    if (i + 1 < Lx) atomicAdd(row + i + 1, t);
  }
}

// The pieces of edge P -> Q cut at the grid lines, in order: piece(ax, ay, bx, by, s0,
// s1, i, j) for every piece, s0 and s1 its ends as edge parameters and (i, j) the cell
// that holds it. The cell is tracked across the crossings (the first from the start
// point and the direction, then +-1 per grid line crossed), and the crossings use the
// reciprocals of the edge's extents: GB300's FP64 rate makes divisions and floors per
// piece the bulk of the rasteriser's work.
template <typename F>
__device__ __forceinline__ void edge_pieces(double2 P, double2 Q, int Lx, int Ly, F&& piece) {
  const double dx = Q.x - P.x, dy = Q.y - P.y;
  // next grid line crossed along x and along y, as edge parameters in (0, 1]
  double gx = 0.0, gy = 0.0, sx = 2.0, sy = 2.0, rx = 0.0, ry = 0.0;
  const int stx = dx > 0.0 ? 1 : -1, sty = dy > 0.0 ? 1 : -1;
  int i = (int)floor(P.x), j = (int)floor(P.y);
  if (dx != 0.0) {
    if (dx < 0.0) i = (int)ceil(P.x) - 1;
    gx = dx > 0.0 ? (double)(i + 1) : (double)i;
    rx = 1.0 / dx;
    sx = (gx - P.x) * rx;
  }
  if (dy != 0.0) {
    if (dy < 0.0) j = (int)ceil(P.y) - 1;
    gy = dy > 0.0 ? (double)(j + 1) : (double)j;
    ry = 1.0 / dy;
    sy = (gy - P.y) * ry;
  }
  double ax = P.x, ay = P.y, s0 = 0.0;
  const int guard = Lx + Ly + 4;
  for (int it = 0; it < guard; ++it) {
    const double s1 = fmin(fmin(sx, sy), 1.0);
    double bx, by;
    if (s1 >= 1.0) {
      bx = Q.x;
      by = Q.y;
    } else {
      bx = P.x + s1 * dx;
      by = P.y + s1 * dy;
    }
    piece(ax, ay, bx, by, s0, fmin(s1, 1.0), i, j);
    if (s1 >= 1.0) break;
    if (sx <= s1) {
      i += stx;
      gx += (double)stx;
      sx = (gx - P.x) * rx;
    }
    if (sy <= s1) {
      j += sty;
      gy += (double)sty;
      sy = (gy - P.y) * ry;
    }
    ax = bx;
    ay = by;
    s0 = s1;
  }
}

__global__ void raster_edges_kernel(const double2* __restrict__ xy, const int* __restrict__ next,
                                    const int* __restrict__ vreg, const double* __restrict__ w,
                                    double* __restrict__ acc, int Lx, int Ly, int n) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const double wt = w[vreg[v]];
    const double2 P = xy[v], Q = xy[next[v]];
    if (wt == 0.0 || Q.y - P.y == 0.0) continue;
    edge_pieces(P, Q, Lx, Ly, [&](double ax, double ay, double bx, double by, double, double, int i, int j) {
      raster_piece(ax, bx, by - ay, i, j, wt, acc, Lx, Ly);
    });
  }
}

// In-place inclusive prefix sum of every row (one block per row, deterministic order).
__global__ void row_scan_kernel(double* __restrict__ acc, int Lx) {
  __shared__ double wsum[32];
  double* row = acc + (size_t)blockIdx.x * Lx;
  const int nt = blockDim.x;
  const int chunk = Lx / nt;  // Lx is a multiple of blockDim.x
  const int b = threadIdx.x * chunk;
  double s = 0.0;
  for (int k = 0; k < chunk; ++k) s += row[b + k];
  // exclusive scan of the chunk sums across the block
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31 || threadIdx.x == nt - 1) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int nw = (nt + 31) >> 5;
    double v = lane < nw ? wsum[lane] : 0.0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double t = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += t;
    }
    if (lane < nw) wsum[lane] = v;
  }
  __syncthreads();
  double run = incl - s + (warp > 0 ? wsum[warp - 1] : 0.0);
  for (int k = 0; k < chunk; ++k) {
    run += row[b + k];
    row[b + k] = run;
  }
}

// ---------------------------------------------------------------------------
// Areas: per region the signed sum of its rings' shoelace areas (each ring relative to
// its first vertex); then sum(A) and sum(V) in one block; then per region the relative
// error err_r = A_r / A^_r - 1 with A^_r = V_r sum(A) / sum(V), the rasterisation weight
// w_r = A^_r / A_r - 1 and the largest |err_r|. Every sum runs in a fixed order, so the
// results do not vary from run to run. The shoelace sums are split into chunks of at most
// kAreaChunk vertices of one ring (one warp each), so that a region with a long boundary
// does not hold up the whole launch; each region then adds its rings' chunk sums in
// order. GB300's FP64 rate bounds these kernels: the division-heavy last step is spread
// over many blocks.
// ---------------------------------------------------------------------------
__global__ void ring_chunk_kernel(const double2* __restrict__ xy, const long long* __restrict__ off,
                                  const int* __restrict__ chunk_ring, const int* __restrict__ ring_chunk_off,
                                  long long n_chunks, double* __restrict__ chunk_sum) {
  const long long c = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (c >= n_chunks) return;  // whole warps leave together
  const int ring = chunk_ring[c];
  const long long a = off[ring], b = off[ring + 1];
  const long long start = a + (c - ring_chunk_off[ring]) * (long long)kAreaChunk;
  const long long end = min(start + (long long)kAreaChunk, b);
  const double2 o = xy[a];
  double s = 0.0;
  for (long long c0 = start; c0 < end; c0 += 32) {
    // lane l holds the offset of vertex c0 + l from o; its successor's comes from lane
    // l + 1 inside the chunk, and the chunk's last vertex loads it (the successor of the
    // ring's last vertex is o: offset 0)
    const long long v = c0 + lane;
    double2 d = make_double2(0.0, 0.0);
    if (v < end) {
      const double2 p = xy[v];
      d = make_double2(p.x - o.x, p.y - o.y);
    }
    double2 e = make_double2(__shfl_down_sync(0xffffffffu, d.x, 1), __shfl_down_sync(0xffffffffu, d.y, 1));
    if (v < end && (lane == 31 || v + 1 == end)) {
      e = make_double2(0.0, 0.0);
      if (v + 1 < b) {
        const double2 q = xy[v + 1];
        e = make_double2(q.x - o.x, q.y - o.y);
      }
    }
    s += d.x * e.y - e.x * d.y;
  }
  s = warp_sum(s);
  if (lane == 0) chunk_sum[c] = s;
}

// A_r = sum over the region's rings of half their chunk sums (one thread per region).
__global__ void region_area_kernel(const int* __restrict__ reg_off, const int* __restrict__ reg_rings,
                                   const int* __restrict__ ring_chunk_off, const double* __restrict__ chunk_sum,
                                   int R, double* __restrict__ area) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x) {
    double A = 0.0;
    for (int k = reg_off[r]; k < reg_off[r + 1]; ++k) {
      const int ring = reg_rings[k];
      double s = 0.0;
      for (int c = ring_chunk_off[ring]; c < ring_chunk_off[ring + 1]; ++c) s += chunk_sum[c];
      A += 0.5 * s;
    }
    area[r] = A;
  }
}

__device__ __forceinline__ double block_sum_det(double v, double* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  double t = lane < nw ? red[lane] : 0.0;
  t = warp_sum(t);  // every warp computes the same total in the same order
  return t;
}

// sums[0] = sum(A), sums[1] = sum(V); resets the largest error (one block).
__global__ void area_sums_kernel(const double* __restrict__ area, const double* __restrict__ values, int R,
                                 double* __restrict__ sums, IterInfo* info) {
  __shared__ double red[32];
  double sa = 0.0, sv = 0.0;
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    sa += area[r];
    sv += values[r];
  }
  sa = block_sum_det(sa, red);
  sv = block_sum_det(sv, red);
  if (threadIdx.x == 0) {
    sums[0] = sa;
    sums[1] = sv;
    info->max_err = 0.0;
  }
}

__global__ void region_error_kernel(const double* __restrict__ area, const double* __restrict__ values, int R,
                                    const double* __restrict__ sums, double* __restrict__ err,
                                    double* __restrict__ w, IterInfo* info) {
  const double sa = sums[0], sv = sums[1];
  double mx = 0.0;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x) {
    const double target = values[r] * sa / sv;
    const double A = area[r];
    const double e = A / target - 1.0;
    err[r] = e;
    w[r] = target / A - 1.0;
    mx = fmax(mx, fabs(e));  // a NaN error (degenerate area) does not count
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0 && mx > 0.0)
    atomic_max_nonneg(reinterpret_cast<unsigned long long*>(&info->max_err), mx);
}

// Copy the integration's outcome into the per-iteration record.
__global__ void collect_kernel(const DevState* st, IterInfo* info) {
  info->t_end = st->t;
  info->accepted = st->accepted;
  info->rejected = st->rejected;
  info->status = st->status;
  info->loop_ns = global_ns() - st->t_start_ns;
}

// ---------------------------------------------------------------------------
// Points through a projected grid: T(p) = p + bilinear interpolation of the grid
// points' displacements over the quad of cell centres containing p (the nearest quad
// is extended linearly in the half-cell band along the walls). Equal to bilinear
// interpolation of the projected positions, since bilinear interpolation of the cell
// centres themselves reproduces p.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void map_points_kernel(const double2* in, double2* out, long long n,
                                  const V2<T>* __restrict__ disp, int Lx, int Ly, const int* guard) {
  if (guard && *guard < 0) return;  // the outer loop recorded a failed integration
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    const double2 q = in[p];
    const double u = q.x - 0.5, v = q.y - 0.5;
    int i0 = (int)floor(u), j0 = (int)floor(v);
    i0 = i0 < 0 ? 0 : (i0 > Lx - 2 ? Lx - 2 : i0);
    j0 = j0 < 0 ? 0 : (j0 > Ly - 2 ? Ly - 2 : j0);
    const double fx = u - i0, fy = v - j0;
    const size_t k = (size_t)j0 * Lx + i0;
    const V2<T> a = disp[k], b = disp[k + 1], c = disp[k + Lx], d = disp[k + Lx + 1];
    const double gx = 1.0 - fx, gy = 1.0 - fy;
    const double dx = gy * (gx * (double)a.x + fx * (double)b.x) + fy * (gx * (double)c.x + fx * (double)d.x);
    const double dy = gy * (gx * (double)a.y + fx * (double)b.y) + fy * (gx * (double)c.y + fx * (double)d.y);
    out[p] = make_double2(q.x + dx, q.y + dy);
  }
}

}  // namespace cg

namespace cg {

// Signed area of every quad of a projected grid (cell centres + displacements), as the
// cross product of its two edges from the lower-left corner; counts the quads whose area
// is not positive (folds) and the smallest area. out[0]: count (u64), out[1]: bits of the
// smallest area mapped to an order-preserving unsigned key.
__device__ __forceinline__ unsigned long long order_key(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}

template <typename T>
__global__ void fold_kernel(const V2<T>* __restrict__ disp, int Lx, int Ly,
                            unsigned long long* out) {
  __shared__ unsigned long long s_cnt, s_min;
  if (threadIdx.x == 0) {
    s_cnt = 0ull;
    s_min = ~0ull;
  }
  __syncthreads();
  unsigned long long cnt = 0, mn = ~0ull;
  const int nq = (Lx - 1) * (Ly - 1);
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
    const int i = q % (Lx - 1), j = q / (Lx - 1);
    const int k = j * Lx + i;
    const V2<T> d00 = disp[k], d10 = disp[k + 1], d01 = disp[k + Lx];
    const double ax = 1.0 + (double)d10.x - (double)d00.x, ay = (double)d10.y - (double)d00.y;
    const double bx = (double)d01.x - (double)d00.x, by = 1.0 + (double)d01.y - (double)d00.y;
    const double area = ax * by - ay * bx;
    if (!(area > 0.0)) ++cnt;
    const unsigned long long key = order_key(area);
    mn = key < mn ? key : mn;
  }
  atomicAdd(&s_cnt, cnt);
  atomicMin(&s_min, mn);
  __syncthreads();
  if (threadIdx.x == 0) {
    atomicAdd(&out[0], s_cnt);
    atomicMin(&out[1], s_min);
  }
}

}  // namespace cg
