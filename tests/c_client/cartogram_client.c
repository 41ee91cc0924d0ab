/* A plain C client of the library's C ABI (include/cartogram.h), with no Python and no
 * CUDA headers: two vertical strips of a 64 x 16 grid with target values 1 and 3. Their
 * density depends on x alone, so the equalising map is the one-dimensional one (main
 * text, the cumulative-density construction): the shared edge at x = 32 moves to
 * x = 64 * 1 / (1 + 3) = 16. Runs both precisions; prints one line per run and returns
 * 0 when both converge with the edge within 1% of the box width of x = 16. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "cartogram.h"

/* counter-clockwise rectangle, sides cut into pieces of at most `step` */
static int rect(double x0, double y0, double x1, double y1, double step, double* xy) {
  const double cx[4] = {x0, x1, x1, x0}, cy[4] = {y0, y0, y1, y1};
  int n = 0;
  for (int k = 0; k < 4; ++k) {
    const double ax = cx[k], ay = cy[k], bx = cx[(k + 1) % 4], by = cy[(k + 1) % 4];
    const int pieces = (int)ceil(hypot(bx - ax, by - ay) / step - 1e-12);
    for (int s = 0; s < pieces; ++s) {
      xy[2 * n] = ax + (bx - ax) * s / pieces;
      xy[2 * n + 1] = ay + (by - ay) * s / pieces;
      ++n;
    }
  }
  return n;
}

static int run(int precision) {
  const int Lx = 64, Ly = 16;
  double* xy = (double*)malloc(sizeof(double) * 2 * 1024);
  int64_t off[3];
  int32_t reg[2] = {0, 1};
  off[0] = 0;
  off[1] = rect(0.0, 0.0, 32.0, Ly, 1.0, xy);
  off[2] = off[1] + rect(32.0, 0.0, Lx, Ly, 1.0, xy + 2 * off[1]);
  const double values[2] = {1.0, 3.0};
  double* x0 = (double*)malloc(sizeof(double) * off[2]);
  for (int64_t v = 0; v < off[2]; ++v) x0[v] = xy[2 * v];
  cg_options opt;
  cartogram_default_options(&opt);
  opt.precision = precision;
  cg_ctx* ctx = NULL;
  int rc = cartogram_init(Lx, Ly, 0.0, &opt, &ctx);
  if (rc != CG_OK) {
    printf("init failed: %d\n", rc);
    free(xy);
    free(x0);
    return rc;
  }
  cg_stats st;
  rc = cartogram_set_regions(ctx, 2, values, 2, off, reg, xy);
  if (rc == CG_OK) rc = cartogram_integrate(ctx, &st);
  double err[2] = {0.0, 0.0}, edge = 1e300;
  if (rc == CG_OK) rc = cartogram_area_errors(ctx, err);
  if (rc == CG_OK) rc = cartogram_get_vertices(ctx, xy);
  if (rc == CG_OK) {
    /* the first strip's right side: its vertices with x = 32 before the run */
    double worst = 0.0;
    for (int64_t v = 0; v < off[1]; ++v)
      if (x0[v] == 32.0) worst = fmax(worst, fabs(xy[2 * v] - 16.0));
    edge = worst;
  }
  if (rc != CG_OK) {
    printf("precision %d failed: %d (%s)\n", precision, rc, cartogram_last_error(ctx));
  } else {
    printf("precision %d: iterations %d, max area error %.3g, edge off by %.3g cells\n", precision, st.iterations,
           fmax(fabs(err[0]), fabs(err[1])), edge);
    if (!st.converged || fabs(err[0]) >= 0.01 || fabs(err[1]) >= 0.01 || edge >= 0.01 * Lx) rc = -100;
  }
  cartogram_destroy(ctx);
  free(xy);
  free(x0);
  return rc;
}

int main(void) {
  const int a = run(CG_PRECISION_FP64), b = run(CG_PRECISION_MIXED);
  if (a != CG_OK || b != CG_OK) return 1;
  printf("ok\n");
  return 0;
}
