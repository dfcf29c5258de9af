// Quadrature nodes of the interior-density face integral (Sec. 4.1,
// Eq. IntDens) that stay accurate when the evaluation point r is close to the
// face.  The face is split at the foot F of r (height h above the face) into
// three signed triangles (F, A, B), one per edge, and each is integrated in
// polar coordinates seen from r: the azimuth psi about the face normal, from
// the direction of A - F to that of B - F, and the polar angle phi from the
// normal up to the edge, phi in [0, atan(l(psi) / h)] with l(psi) the distance
// from F to the edge along psi.  In these variables the area element times
// cos(theta) / R^2 is sin(phi) dphi dpsi, so the integrand (with exp(-mu R)
// and the Zernike vector of the direction) is smooth and tensor
// Gauss-Legendre converges fast where a rule on the flat triangle does not.
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

// Node k in [0, 3 n^2) of the split polar rule for face (P0, P1, P2) with
// inward unit normal nin and frame (e1, e2), evaluation point r (inside the
// tet, h > 0).  gx, gw: n-point Gauss-Legendre nodes and weights on [-1, 1].
// k = (edge * n + a) * n + b: edge of the face, azimuth node a, polar node b.
// A degenerate triangle (F on an edge's line) gives weight 0.
DFM_HD inline PolarNode polar_node(const double P[3][3], const double nin[3], const double e1[3],
                                   const double e2[3], const double r[3], int n, int k, const double* gx,
                                   const double* gw) {
  PolarNode out = {0.0, 1.0, 0.0, 0.0};
  const int edge = k / (n * n);
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
  const double dpsi = atan2(Ax * By - Ay * Bx, Ax * Bx + Ay * By);  // signed angle from A to B
  if (fabs(dpsi) < 1e-15) return out;
  const double xa = 0.5 * (gx[a] + 1.0), wa = 0.5 * gw[a];
  const double xb = 0.5 * (gx[b] + 1.0), wb = 0.5 * gw[b];
  const double psi = atan2(Ay, Ax) + xa * dpsi;
  const double ex = cos(psi), ey = sin(psi);
  const double ABx = Bx - Ax, ABy = By - Ay;
  const double den = ex * ABy - ey * ABx;
  if (den == 0.0) return out;
  const double ell = (Ax * ABy - Ay * ABx) / den;  // F + ell (ex, ey) lies on the edge's line
  const double Phi = atan2(ell, h);
  const double phi = Phi * xb;
  const double sphi = sin(phi);
  out.w = orient * wa * dpsi * Phi * wb * sphi;
  out.R = h / cos(phi);
  out.dx = -sphi * ex;
  out.dy = -sphi * ey;
  return out;
}

}  // namespace rule
}  // namespace dfm
