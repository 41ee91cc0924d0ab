// Diagnostics of the composed projection T = T_K o ... o T_1 (T_k: bilinear
// interpolation of iteration k's projected grid over the quads of cell centres, the
// nearest quad extended across the half-cell band along the walls -- the map that
// maps the vertices):
//  - angular distortion (SI section 3, Tissot indicatrix): e = ln(a/b) and
//    e~ = 2 asin((a - b)/(a + b)) from the singular values a >= b of the Jacobian of T,
//    averaged and maximised over the quad centres of the original lattice;
//  - the inverse map (the main text's inverse graticule): preimages of points under T,
//    grid by grid in reverse order.
// Both work in FP64 on the stored displacements.
#pragma once

#include "common.cuh"

namespace cg {

// Quad (i0, j0) of the cell-centre lattice that a grid's map uses at (x, y), and the
// fractional position (fx, fy) in it (outside [0, 1] in the wall bands).
__device__ __forceinline__ void locate_quad(int Lx, int Ly, double x, double y, int& i0, int& j0, double& fx,
                                            double& fy) {
  const double u = x - 0.5, w = y - 0.5;
  const double fu = floor(fmin(fmax(u, -1.0), (double)Lx)), fw = floor(fmin(fmax(w, -1.0), (double)Ly));
  i0 = min(max((int)fu, 0), Lx - 2);
  j0 = min(max((int)fw, 0), Ly - 2);
  fx = u - i0;
  fy = w - j0;
}

// Corner displacements of quad (i0, j0) of grid `g` (promoted to FP64).
template <typename T>
__device__ __forceinline__ void quad_corners(const V2<T>* __restrict__ g, int Lx, int i0, int j0, double2 (&q)[4]) {
  const size_t k00 = (size_t)j0 * Lx + i0;
  const V2<T> a = g[k00], b = g[k00 + 1], c = g[k00 + Lx], d = g[k00 + Lx + 1];
  q[0] = make_double2(a.x, a.y);
  q[1] = make_double2(b.x, b.y);
  q[2] = make_double2(c.x, c.y);
  q[3] = make_double2(d.x, d.y);
}

// e and e~ at the centre of every quad of the original lattice; per-block sums into
// part[2 * block] (e, e~) and maxima into max_bits[0..1] (bit patterns of
// non-negative doubles).
template <typename T>
__global__ void __launch_bounds__(256) distortion_kernel(const void* const* __restrict__ hist, int K, int Lx,
                                                         int Ly, double* __restrict__ part,
                                                         unsigned long long* max_bits) {
  __shared__ double s_e[256], s_t[256];
  const int M = (Lx - 1) * (Ly - 1);
  double se = 0.0, st = 0.0, me = 0.0, mt = 0.0;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < M; p += gridDim.x * blockDim.x) {
    const int i = p % (Lx - 1), j = p / (Lx - 1);
    double x = i + 1.0, y = j + 1.0;
    double a = 1.0, b = 0.0, c = 0.0, d = 1.0;  // J = [[a, b], [c, d]]
    for (int k = 0; k < K; ++k) {
      const V2<T>* g = reinterpret_cast<const V2<T>*>(hist[k]);
      int i0, j0;
      double fx, fy;
      locate_quad(Lx, Ly, x, y, i0, j0, fx, fy);
      double2 q[4];
      quad_corners<T>(g, Lx, i0, j0, q);
      // projected corners P = centre + displacement; the centres' own differences are
      // the unit steps of the lattice
      const double txx = 1.0 + (1 - fy) * (q[1].x - q[0].x) + fy * (q[3].x - q[2].x);
      const double tyx = (1 - fy) * (q[1].y - q[0].y) + fy * (q[3].y - q[2].y);
      const double txy = (1 - fx) * (q[2].x - q[0].x) + fx * (q[3].x - q[1].x);
      const double tyy = 1.0 + (1 - fx) * (q[2].y - q[0].y) + fx * (q[3].y - q[1].y);
      const double na = txx * a + txy * c, nb = txx * b + txy * d;
      const double nc = tyx * a + tyy * c, nd = tyx * b + tyy * d;
      a = na;
      b = nb;
      c = nc;
      d = nd;
      const double c00 = (1 - fx) * (1 - fy), c10 = fx * (1 - fy), c01 = (1 - fx) * fy, c11 = fx * fy;
      x += c00 * q[0].x + c10 * q[1].x + c01 * q[2].x + c11 * q[3].x;
      y += c00 * q[0].y + c10 * q[1].y + c01 * q[2].y + c11 * q[3].y;
    }
    // singular values from the conformal and anti-conformal parts of J
    const double pp = hypot(a + d, c - b), qq = hypot(a - d, c + b);
    const double s1 = 0.5 * (pp + qq), s2 = 0.5 * fabs(pp - qq);
    const double e = log(s1 / s2), et = 2.0 * asin((s1 - s2) / (s1 + s2));
    se += e;
    st += et;
    me = fmax(me, e);
    mt = fmax(mt, et);
  }
  s_e[threadIdx.x] = se;
  s_t[threadIdx.x] = st;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      s_e[threadIdx.x] += s_e[threadIdx.x + w];
      s_t[threadIdx.x] += s_t[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = s_e[0];
    part[2 * blockIdx.x + 1] = s_t[0];
  }
  me = warp_max(me);
  mt = warp_max(mt);
  if ((threadIdx.x & 31) == 0) {
    atomic_max_nonneg(&max_bits[0], me);
    atomic_max_nonneg(&max_bits[1], mt);
  }
}

// Sums of the per-block parts in a fixed order, and the means (one thread).
static __global__ void distortion_finish_kernel(const double* part, int nblocks, const unsigned long long* max_bits,
                                                int M, double* out) {
  double se = 0.0, st = 0.0;
  for (int b = 0; b < nblocks; ++b) {
    se += part[2 * b];
    st += part[2 * b + 1];
  }
  out[0] = se / M;
  out[1] = __longlong_as_double((long long)max_bits[0]);
  out[2] = st / M;
  out[3] = __longlong_as_double((long long)max_bits[1]);
}

// Preimage of (qx, qy) under one grid's map. The bilinear map of a quad sends its
// domain's edges to straight segments, so the image of the domain is the quadrilateral
// of its corners' images: q is located by walking from quad to quad across the edge
// that q lies beyond (the domains of the quads along the walls extend to the box edge),
// then Newton's method on the quad's bilinear map gives the position. false if q lies
// outside the image of the box or the walk does not settle within its step limit.
template <typename T>
__device__ bool invert_grid(const V2<T>* __restrict__ g, int Lx, int Ly, double qx, double qy, double& px,
                            double& py) {
  // start in the quad of q shifted back by the displacement found there
  int i0, j0;
  double fx, fy;
  locate_quad(Lx, Ly, qx, qy, i0, j0, fx, fy);
  {
    double2 q[4];
    quad_corners<T>(g, Lx, i0, j0, q);
    const double c00 = (1 - fx) * (1 - fy), c10 = fx * (1 - fy), c01 = (1 - fx) * fy, c11 = fx * fy;
    const double gx = qx - (c00 * q[0].x + c10 * q[1].x + c01 * q[2].x + c11 * q[3].x);
    const double gy = qy - (c00 * q[0].y + c10 * q[1].y + c01 * q[2].y + c11 * q[3].y);
    locate_quad(Lx, Ly, gx, gy, i0, j0, fx, fy);
  }
  const int max_walk = 4 * (Lx + Ly);
  for (int step = 0; step < max_walk; ++step) {
    double2 q[4];
    quad_corners<T>(g, Lx, i0, j0, q);
    // projected corners of the quad
    const double x00 = i0 + 0.5 + q[0].x, y00 = j0 + 0.5 + q[0].y;
    const double x10 = i0 + 1.5 + q[1].x, y10 = j0 + 0.5 + q[1].y;
    const double x01 = i0 + 0.5 + q[2].x, y01 = j0 + 1.5 + q[2].y;
    const double x11 = i0 + 1.5 + q[3].x, y11 = j0 + 1.5 + q[3].y;
    auto bil = [&](double u, double v, double& x, double& y) {
      x = (1 - u) * (1 - v) * x00 + u * (1 - v) * x10 + (1 - u) * v * x01 + u * v * x11;
      y = (1 - u) * (1 - v) * y00 + u * (1 - v) * y10 + (1 - u) * v * y01 + u * v * y11;
    };
    const double ulo = i0 == 0 ? -0.5 : 0.0, uhi = i0 == Lx - 2 ? 1.5 : 1.0;
    const double vlo = j0 == 0 ? -0.5 : 0.0, vhi = j0 == Ly - 2 ? 1.5 : 1.0;
    // image of the domain: corners A (lo, lo), B (hi, lo), C (hi, hi), D (lo, hi)
    double ax, ay, bx, by, cx, cy, dx, dy;
    bil(ulo, vlo, ax, ay);
    bil(uhi, vlo, bx, by);
    bil(uhi, vhi, cx, cy);
    bil(ulo, vhi, dx, dy);
    const double area = (bx - ax) * (dy - ay) - (by - ay) * (dx - ax) + (dx - cx) * (by - cy) - (dy - cy) * (bx - cx);
    const double sg = area >= 0.0 ? 1.0 : -1.0;
    const double tol = 1e-12 * (fabs(area) + 1.0);
    const bool below = sg * ((bx - ax) * (qy - ay) - (by - ay) * (qx - ax)) < -tol;
    const bool right = sg * ((cx - bx) * (qy - by) - (cy - by) * (qx - bx)) < -tol;
    const bool above = sg * ((dx - cx) * (qy - cy) - (dy - cy) * (qx - cx)) < -tol;
    const bool left = sg * ((ax - dx) * (qy - dy) - (ay - dy) * (qx - dx)) < -tol;
    const int mi = right ? 1 : (left ? -1 : 0), mj = above ? 1 : (below ? -1 : 0);
    if (mi == 0 && mj == 0) {
      double u = 0.5 * (ulo + uhi), v = 0.5 * (vlo + vhi);
      for (int it = 0; it < 40; ++it) {
        double x, y;
        bil(u, v, x, y);
        const double rx = x - qx, ry = y - qy;
        const double xu = (1 - v) * (x10 - x00) + v * (x11 - x01), yu = (1 - v) * (y10 - y00) + v * (y11 - y01);
        const double xv = (1 - u) * (x01 - x00) + u * (x11 - x10), yv = (1 - u) * (y01 - y00) + u * (y11 - y10);
        const double det = xu * yv - xv * yu;
        if (!(fabs(det) > 0.0)) return false;
        const double du = (rx * yv - ry * xv) / det, dv = (ry * xu - rx * yu) / det;
        u -= du;
        v -= dv;
        if (!(fabs(u) < 1e3 && fabs(v) < 1e3)) return false;
        if (fabs(du) + fabs(dv) < 1e-15) break;
      }
      double x, y;
      bil(u, v, x, y);
      if (!(fabs(x - qx) + fabs(y - qy) < 1e-9)) return false;
      px = i0 + 0.5 + u;
      py = j0 + 0.5 + v;
      return true;
    }
    const int ni = min(max(i0 + mi, 0), Lx - 2), nj = min(max(j0 + mj, 0), Ly - 2);
    if (ni == i0 && nj == j0) return false;  // beyond the image of the box
    i0 = ni;
    j0 = nj;
  }
  return false;
}

// Preimages of n points under the composed projection (NaN where none is found).
template <typename T>
__global__ void inverse_points_kernel(const void* const* __restrict__ hist, int K, int Lx, int Ly, long long n,
                                      double2* pts) {
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    double x = pts[p].x, y = pts[p].y;
    bool ok = true;
    for (int k = K - 1; k >= 0 && ok; --k) {
      double px = 0.0, py = 0.0;
      ok = invert_grid<T>(reinterpret_cast<const V2<T>*>(hist[k]), Lx, Ly, x, y, px, py);
      x = px;
      y = py;
    }
    pts[p] = ok ? make_double2(x, y) : make_double2(__longlong_as_double(0x7ff8000000000000ll),
                                                    __longlong_as_double(0x7ff8000000000000ll));
  }
}

// ---------------------------------------------------------------------------
// Polygon-level measures (SI section 4): the mean aspect ratio of the regions' minimum-
// area bounding rectangles, and the relative position error of their centroids between
// two vertex sets (the input map and the current one). A region's points are the vertices
// of all its rings.
// ---------------------------------------------------------------------------

// Centroids of the regions from the shoelace moments of their rings (signed: holes
// subtract), one warp per region.
__global__ void region_centroid_kernel(const double2* __restrict__ xy, const long long* __restrict__ off,
                                       const int* __restrict__ reg_off, const int* __restrict__ reg_rings, int R,
                                       double2* __restrict__ cent) {
  const int r = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= R) return;  // whole warps leave together
  double A = 0.0, Mx = 0.0, My = 0.0;
  for (int k = reg_off[r]; k < reg_off[r + 1]; ++k) {
    const int ring = reg_rings[k];
    const long long a = off[ring], b = off[ring + 1];
    for (long long v = a + lane; v < b; v += 32) {
      const double2 p = xy[v], q = xy[v + 1 < b ? v + 1 : a];
      const double cr = p.x * q.y - q.x * p.y;
      A += cr;
      Mx += (p.x + q.x) * cr;
      My += (p.y + q.y) * cr;
    }
  }
  A = warp_sum(A);
  Mx = warp_sum(Mx);
  My = warp_sum(My);
  // (M / 6) / (A / 2)
  if (lane == 0) cent[r] = make_double2(Mx / (3.0 * A), My / (3.0 * A));
}

// Sum over the pairs i < j of the angle between c_i - c_j and d_i - d_j (atan2 of the
// cross product's magnitude and the dot product: the arccos of their cosine without its
// loss of accuracy near 0 and pi; 0 where a vector vanishes); block b covers the rows
// i = b, b + gridDim.x, ... and writes its sum to part[b] (fixed order within the block).
__global__ void position_error_kernel(const double2* __restrict__ c, const double2* __restrict__ d, int R,
                                      double* __restrict__ part) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int i = blockIdx.x; i < R - 1; i += gridDim.x) {
    const double2 ci = c[i], di = d[i];
    for (int j = i + 1 + threadIdx.x; j < R; j += blockDim.x) {
      const double ux = ci.x - c[j].x, uy = ci.y - c[j].y;
      const double wx = di.x - d[j].x, wy = di.y - d[j].y;
      // products rounded on their own (no fused multiply-add): the cross product of two
      // equal vectors is then exactly 0
      acc += atan2(fabs(__dmul_rn(ux, wy) - __dmul_rn(uy, wx)), __dmul_rn(ux, wx) + __dmul_rn(uy, wy));
    }
  }
  acc = warp_sum(acc);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}

// Gift wrapping needs "the point q such that no point lies right of p -> q"; between two
// candidates a and b the one more clockwise about p wins, and of collinear ones the
// farther (so that points on a hull edge are skipped). Collinear means within 1e-12 of
// |a - p| |b - p|: the subdivided straight edges of a map put hundreds of points on a line
// to within rounding, where the exact sign of the cross product is noise and would make
// the comparison inconsistent (the march could then wander instead of closing).
__device__ __forceinline__ bool wrap_better(double2 p, double2 a, double2 b) {
  const double ax = a.x - p.x, ay = a.y - p.y, bx = b.x - p.x, by = b.y - p.y;
  const double da = ax * ax + ay * ay, db = bx * bx + by * by;
  const double cr = ax * by - ay * bx, tol = 1e-12 * sqrt(da * db);
  if (cr < -tol) return true;  // b lies right of p -> a
  if (cr > tol) return false;
  return db > da;
}

constexpr int kHullMax = 2048;
constexpr double kRectTie = 1e-9;  // rectangle areas this close (relative) are the same minimum

// Area and aspect ratio of the bounding rectangle of the convex polygon hull[0..h) with a
// side along edge e.
__device__ __forceinline__ void hull_rectangle(const double2* hull, int h, int e, double& area, double& ratio) {
  const double2 a = hull[e], b = hull[e + 1 < h ? e + 1 : 0];
  const double len = sqrt((b.x - a.x) * (b.x - a.x) + (b.y - a.y) * (b.y - a.y));
  const double ux = (b.x - a.x) / len, uy = (b.y - a.y) / len;
  double lo1 = INFINITY, hi1 = -INFINITY, lo2 = INFINITY, hi2 = -INFINITY;
  for (int k = 0; k < h; ++k) {
    const double2 q = hull[k];
    const double s1 = q.x * ux + q.y * uy, s2 = q.y * ux - q.x * uy;
    lo1 = fmin(lo1, s1);
    hi1 = fmax(hi1, s1);
    lo2 = fmin(lo2, s2);
    hi2 = fmax(hi2, s2);
  }
  const double w = hi1 - lo1, t = hi2 - lo2;
  area = w * t;
  ratio = fmax(w, t) / fmin(w, t);
}

// Aspect ratio alpha_r of every region: its convex hull by gift wrapping (each step one
// block-wide scan of the region's points), then the bounding rectangle along every hull
// edge (the minimum-area rectangle of a convex polygon has a side on one of its edges);
// the smallest area wins, exact ties to the smaller ratio. One block per region (grid-
// stride); a hull of more than kHullMax vertices gives NaN.
__global__ void aspect_ratio_kernel(const double2* __restrict__ xy, const long long* __restrict__ off,
                                    const int* __restrict__ reg_off, const int* __restrict__ reg_rings, int R,
                                    double* __restrict__ alpha) {
  __shared__ double2 hull[kHullMax];
  __shared__ double2 s_pt[32];
  __shared__ double s_a[32], s_r[32];
  __shared__ int s_h, s_done;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int r = blockIdx.x; r < R; r += gridDim.x) {
    const int k0 = reg_off[r], k1 = reg_off[r + 1];
    // the lowest point (smallest x, then y) is on the hull
    double2 best = make_double2(INFINITY, INFINITY);
    for (int k = k0; k < k1; ++k) {
      const long long a = off[reg_rings[k]], b = off[reg_rings[k] + 1];
      for (long long v = a + threadIdx.x; v < b; v += blockDim.x) {
        const double2 q = xy[v];
        if (q.x < best.x || (q.x == best.x && q.y < best.y)) best = q;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double2 q = make_double2(__shfl_xor_sync(0xffffffffu, best.x, o), __shfl_xor_sync(0xffffffffu, best.y, o));
      if (q.x < best.x || (q.x == best.x && q.y < best.y)) best = q;
    }
    if (lane == 0) s_pt[warp] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
      double2 b0 = s_pt[0];
      for (int w = 1; w < nw; ++w) {
        const double2 q = s_pt[w];
        if (q.x < b0.x || (q.x == b0.x && q.y < b0.y)) b0 = q;
      }
      hull[0] = b0;
      s_h = 1;
      s_done = 0;
    }
    __syncthreads();
    const double2 start = hull[0];
    // gift wrapping: at most kHullMax steps
    for (int it = 0; it < kHullMax; ++it) {
      const double2 p = hull[s_h - 1];
      double2 cand = p;
      bool have = false;
      for (int k = k0; k < k1; ++k) {
        const long long a = off[reg_rings[k]], b = off[reg_rings[k] + 1];
        for (long long v = a + threadIdx.x; v < b; v += blockDim.x) {
          const double2 q = xy[v];
          if (q.x == p.x && q.y == p.y) continue;
          if (!have || wrap_better(p, cand, q)) {
            cand = q;
            have = true;
          }
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double2 q = make_double2(__shfl_xor_sync(0xffffffffu, cand.x, o), __shfl_xor_sync(0xffffffffu, cand.y, o));
        const bool qh = __shfl_xor_sync(0xffffffffu, have ? 1 : 0, o) != 0;
        if (qh && (!have || wrap_better(p, cand, q))) {
          cand = q;
          have = true;
        }
      }
      if (lane == 0) s_pt[warp] = have ? cand : make_double2(NAN, NAN);
      __syncthreads();
      if (threadIdx.x == 0) {
        double2 q0 = make_double2(NAN, NAN);
        for (int w = 0; w < nw; ++w) {
          const double2 q = s_pt[w];
          if (q.x != q.x) continue;  // no candidate in that warp
          if (q0.x != q0.x || wrap_better(p, q0, q)) q0 = q;
        }
        if (q0.x != q0.x || (q0.x == start.x && q0.y == start.y)) s_done = 1;
        else if (s_h < kHullMax) hull[s_h++] = q0;
        else s_done = 2;  // hull too long
      }
      __syncthreads();
      if (s_done) break;
    }
    const int h = s_h;
    const bool too_long = s_done == 2;
    // the rectangle along every hull edge: the smallest area, then the smallest ratio among
    // the edges whose area is within kRectTie of it (two orientations often tie, and the
    // ratio jumps between them: rounding must not pick the side)
    double ba = INFINITY;
    for (int pass = 0; pass < 2; ++pass) {
      double bv = INFINITY;
      for (int e = threadIdx.x; e < h && h >= 3; e += blockDim.x) {
        double area, ratio;
        hull_rectangle(hull, h, e, area, ratio);
        if (pass == 0) bv = fmin(bv, area);
        else if (area <= ba * (1.0 + kRectTie)) bv = fmin(bv, ratio);
      }
      for (int o = 16; o > 0; o >>= 1) bv = fmin(bv, __shfl_xor_sync(0xffffffffu, bv, o));
      if (lane == 0) s_a[warp] = bv;
      __syncthreads();
      if (threadIdx.x == 0) {
        double v = s_a[0];
        for (int w = 1; w < nw; ++w) v = fmin(v, s_a[w]);
        s_r[0] = v;
      }
      __syncthreads();
      if (pass == 0) ba = s_r[0];
      __syncthreads();  // s_r[0] is written again by the next pass
    }
    if (threadIdx.x == 0) alpha[r] = (too_long || h < 3) ? NAN : s_r[0];
    __syncthreads();  // the hull is reused by the next region
  }
}

// out[0] = mean of alpha[0..R); with part: out[1] = sum of part[0..nb) * 2 / (R (R - 1) pi)
// (fixed order, one thread).
__global__ void polygon_finish_kernel(const double* __restrict__ alpha, int R, const double* __restrict__ part,
                                      int nb, double* __restrict__ out) {
  double s = 0.0;
  for (int r = 0; r < R; ++r) s += alpha[r];
  out[0] = s / R;
  if (part) {
    double t = 0.0;
    for (int b = 0; b < nb; ++b) t += part[b];
    out[1] = R > 1 ? 2.0 * t / ((double)R * (R - 1) * kPi) : 0.0;
  }
}

}  // namespace cg
