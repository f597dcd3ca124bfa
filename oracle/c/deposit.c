/* FP64 mesh assignment for the oracle (TEST INFRASTRUCTURE ONLY).
 *
 * Same definitions as oracle/assignment.py, written as a plain loop so that the
 * survey-sized catalogues (tens of millions of particles) can be deposited in
 * seconds: u = (x - box_min)/H - shift per axis (FP64 from the float32 input),
 *   NGP: node floor(u + 1/2), weight 1
 *   CIC: nodes floor(u), floor(u) + 1 with weights 1 - d, d  (d = u - floor(u))
 *   TSC: c = floor(u + 1/2), d = u - c; nodes c - 1, c, c + 1 with weights
 *        (1/2)(1/2 - d)^2, 3/4 - d^2, (1/2)(1/2 + d)^2
 * indices taken mod N, mesh[(ix * N + iy) * N + iz] += w * wx * wy * wz.
 */
#include <math.h>
#include <stdint.h>

static int stencil(double u, int kind, long *node, double *wt) {
  if (kind == 1) {
    node[0] = (long)floor(u + 0.5);
    wt[0] = 1.0;
    return 1;
  }
  if (kind == 2) {
    double i = floor(u), d = u - i;
    node[0] = (long)i; node[1] = (long)i + 1;
    wt[0] = 1.0 - d; wt[1] = d;
    return 2;
  }
  double c = floor(u + 0.5), d = u - c;
  node[0] = (long)c - 1; node[1] = (long)c; node[2] = (long)c + 1;
  wt[0] = 0.5 * (0.5 - d) * (0.5 - d);
  wt[1] = 0.75 - d * d;
  wt[2] = 0.5 * (0.5 + d) * (0.5 + d);
  return 3;
}

static long wrap(long v, long n) {
  long r = v % n;
  return r < 0 ? r + n : r;
}

void oracle_deposit(const float *x, const float *y, const float *z, const double *w, int64_t n,
                    const double *box_min, double H, int N, int kind, double shift, double *mesh) {
  for (int64_t p = 0; p < n; ++p) {
    const float *c3[3] = {x, y, z};
    long node[3][3];
    double wt[3][3];
    int cnt = 0;
    for (int a = 0; a < 3; ++a) {
      double u = ((double)c3[a][p] - box_min[a]) / H - shift;
      cnt = stencil(u, kind, node[a], wt[a]);
    }
    for (int i = 0; i < cnt; ++i) {
      long jx = wrap(node[0][i], N);
      for (int j = 0; j < cnt; ++j) {
        long jy = wrap(node[1][j], N);
        double wxy = w[p] * wt[0][i] * wt[1][j];
        for (int k = 0; k < cnt; ++k) {
          long jz = wrap(node[2][k], N);
          mesh[(jx * N + jy) * N + jz] += wxy * wt[2][k];
        }
      }
    }
  }
}
