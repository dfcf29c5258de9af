// Quadrature nodes of the interior-density face integral (Sec. 4.1,
// Eq. IntDens) that stay accurate when the evaluation point r is close to the
// face, or its foot F on the face plane is close to an edge (thin tets of a
// jittered mesh have both).  The face is split at F (height h above the face)
// into three signed triangles (F, A, B), one per edge, and each is integrated
// in polar coordinates seen from r: the azimuth about the face normal and the
// polar angle phi from the normal up to the edge, phi in [0, atan(l / h)] with
// l the distance from F to the edge point X hit at that azimuth.  In these
// variables the area element times cos(theta) / R^2 is sin(phi) dphi dpsi.
// The azimuth is not sampled uniformly: the edge point X = M + u t (M the
// foot of the perpendicular from F to the edge's line, t the unit edge
// direction, d = |F M|) is, with dpsi = d du / (d^2 + u^2) and
// u = c tan(s), c = sqrt(h^2 + d^2), and Gauss-Legendre nodes uniform in s;
// each edge is cut in two pieces at M (or at its middle in s when M lies
// outside the edge).  The integrand in u varies on the scale c, so it stays
// smooth in s both when F is close to the edge's line (d << h, where a rule
// uniform in the azimuth needs many more nodes) and when r is close to the
// face (h << d, where s is the azimuth itself); tensor Gauss-Legendre in s
// and in phi converges fast.
//
// Plain arithmetic with no CUDA intrinsics, so the same function serves the
// device kernel and a host-side check of the nodes.
#pragma once

#include <math.h>

#ifdef __CUDACC__
#define DFM_HD __host__ __device__
#else
#define DFM_HD
#endif

namespace dfm {
namespace rule {

struct PolarNode {
  double w;       // weight (sin(phi) dphi dpsi with the Gauss weights and the triangle's sign)
  double R;       // distance from the face point to r
  double dx, dy;  // tangential part of unit(r - s) in the face frame (e1, e2)
};

// Node k in [0, 6 n^2) of the split polar rule for face (P0, P1, P2) with
// inward unit normal nin and frame (e1, e2), evaluation point r (inside the
// tet, h > 0).  gx, gw: n-point Gauss-Legendre nodes and weights on [-1, 1].
// k = ((edge * 2 + piece) * n + a) * n + b: edge of the face, piece of the
// edge, azimuth node a, polar node b.  A degenerate triangle (F on an edge's
// line) gives weight 0.
DFM_HD inline PolarNode polar_node(const double P[3][3], const double nin[3], const double e1[3],
                                   const double e2[3], const double r[3], int n, int k, const double* gx,
                                   const double* gw) {
  PolarNode out = {0.0, 1.0, 0.0, 0.0};
  const int edge = k / (2 * n * n);
  const int piece = (k / (n * n)) & 1;
  const int a = (k / n) % n;
  const int b = k % n;
  double rp[3], u[3], v[3];
  for (int c = 0; c < 3; ++c) rp[c] = r[c] - P[0][c];
  const double h = rp[0] * nin[0] + rp[1] * nin[1] + rp[2] * nin[2];
  double F[3];
  for (int c = 0; c < 3; ++c) F[c] = r[c] - h * nin[c];
  // orientation of the face's vertex order against the inward normal
  for (int c = 0; c < 3; ++c) {
    u[c] = P[1][c] - P[0][c];
    v[c] = P[2][c] - P[0][c];
  }
  const double on = (u[1] * v[2] - u[2] * v[1]) * nin[0] + (u[2] * v[0] - u[0] * v[2]) * nin[1] +
                    (u[0] * v[1] - u[1] * v[0]) * nin[2];
  const double orient = on >= 0.0 ? 1.0 : -1.0;
  // the edge's end points in the face plane, F at the origin
  const double* PA = P[edge];
  const double* PB = P[(edge + 1) % 3];
  double Ax = 0, Ay = 0, Bx = 0, By = 0;
  for (int c = 0; c < 3; ++c) {
    Ax += (PA[c] - F[c]) * e1[c];
    Ay += (PA[c] - F[c]) * e2[c];
    Bx += (PB[c] - F[c]) * e1[c];
    By += (PB[c] - F[c]) * e2[c];
  }
  const double len = sqrt((Bx - Ax) * (Bx - Ax) + (By - Ay) * (By - Ay));
  if (len == 0.0) return out;
  const double tx = (Bx - Ax) / len, ty = (By - Ay) / len;
  const double d = fabs(Ax * ty - Ay * tx);  // distance from F to the edge's line
  if (d < 1e-15 * len) return out;
  const double cr = Ax * By - Ay * Bx;  // sign of the triangle (F, A, B)
  const double sgn = cr > 0.0 ? 1.0 : (cr < 0.0 ? -1.0 : 0.0);
  const double uA = Ax * tx + Ay * ty, uB = Bx * tx + By * ty;
  const double Mx = Ax - uA * tx, My = Ay - uA * ty;  // foot of the perpendicular from F
  const double cc = sqrt(h * h + d * d);
  const double sA = atan2(uA, cc), sB = atan2(uB, cc);
  const double cut = (sA < 0.0 && sB > 0.0) ? 0.0 : 0.5 * (sA + sB);
  const double s0 = piece ? cut : sA, s1 = piece ? sB : cut;
  const double xa = 0.5 * (gx[a] + 1.0), wa = 0.5 * gw[a];
  const double xb = 0.5 * (gx[b] + 1.0), wb = 0.5 * gw[b];
  const double sv = s0 + (s1 - s0) * xa;
  const double cs = cos(sv);
  const double uu = cc * tan(sv);
  const double ell = sqrt(d * d + uu * uu);
  const double ex = (Mx + uu * tx) / ell, ey = (My + uu * ty) / ell;  // unit direction from F to the edge point
  // dpsi = d du / ell^2, du = c ds / cos^2(s)
  const double jac = (s1 - s0) * wa * cc / (cs * cs) * d / (ell * ell);
  const double Phi = atan2(ell, h);
  const double phi = Phi * xb;
  const double sphi = sin(phi);
  out.w = orient * sgn * jac * Phi * wb * sphi;
  out.R = h / cos(phi);
  out.dx = -sphi * ex;
  out.dy = -sphi * ey;
  return out;
}

}  // namespace rule
}  // namespace dfm
