/*
 * FP64 CPU oracle for discrete flow mapping (DFM) on tetrahedral meshes.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may call this code; the product path never
 * does.  It shares no code with the CUDA library.
 *
 * What it computes (Bajars, Chappell, Sondergaard, Tanner, "Transport of
 * phase space densities through tetrahedral meshes using discrete flow
 * mapping"):
 *
 *   B_IJ = lambda * N_{n'm'} / sqrt(|T_l| |T_l'|)
 *          * Int_{hemisphere} Z_{n'}^{m'}(p') Z_n^m(p) S_{l->l'}(d) cos(theta) dw
 *
 * (Sec. 3.2, Eqs. Bapprox and B4DInt with rho = sin(theta), so that
 * rho drho dphi = cos(theta) dw), where S_{l->l'}(d) is the damped area of the
 * set of source points on face l whose ray in direction d leaves the tet
 * through face l' (Sec. 3.3), N_{n'm'} = (2n'+2)/(eps_{m'} pi) is the inverse
 * Zernike norm (Sec. 3.1) and lambda the reflection/transmission weight.
 *
 * Routes chosen to be independent of the GPU path:
 *   - Zernike radial polynomials by the factorial closed form and angles by
 *     atan2/cos/sin (the GPU uses the recursion of Sec. 3.1);
 *   - S_{l->l'}(d) by projecting face l' onto the plane of face l along d,
 *     clipping against face l (Sutherland-Hodgman) and integrating exp(-mu L)
 *     over the clipped polygon with a collapsed Gauss rule (the GPU uses the
 *     closed form of Sec. 3.3 on the triangle OBC);
 *   - the direction integral over the seven sub-regions of Sec. 3.4, each
 *     mapped from [-1,1]^2 by the bilinear map of Eq. (Parametr) and projected
 *     onto the hemisphere, with tensor Gauss-Legendre nodes supplied by the
 *     caller (numpy) and the order doubled until successive estimates agree.
 *
 * Conventions (the paper leaves the face frame open, Sec. 3.3): tet t has
 * vertices (v0,v1,v2,v3); face f is opposite v_f with vertices
 * (v_{f+1}, v_{f+2}, v_{f+3}) mod 4; row 4t+f.  Frame origin = first face
 * vertex, e1 = unit(second - first), n = inward unit normal (towards v_f),
 * e2 = n x e1.  Momentum p = (d.e1, d.e2) for inward unit direction d.
 * Zernike index idx = (n(n+2)+m)/2, m = -n, -n+2, ..., n.
 */
#include <math.h>

/* Planted mistakes for the mutation test of the pins: the tests build this file
 * a second time with -DORC_MUTATE=k and check that some pin fails; the oracle
 * itself is built with the default 0, which compiles none of them. */
#ifndef ORC_MUTATE
#define ORC_MUTATE 0
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct { double x, y, z; } vec3;

static vec3 v3(double x, double y, double z) { vec3 r = {x, y, z}; return r; }
static vec3 vadd(vec3 a, vec3 b) { return v3(a.x + b.x, a.y + b.y, a.z + b.z); }
static vec3 vsub(vec3 a, vec3 b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
static vec3 vscale(vec3 a, double s) { return v3(a.x * s, a.y * s, a.z * s); }
static double vdot(vec3 a, vec3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static vec3 vcross(vec3 a, vec3 b) {
  return v3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static double vnorm(vec3 a) { return sqrt(vdot(a, a)); }
static vec3 vunit(vec3 a) { return vscale(a, 1.0 / vnorm(a)); }

static vec3 vert(const double* V, int64_t i) { return v3(V[3 * i], V[3 * i + 1], V[3 * i + 2]); }

/* ------------------------------------------------------------------------ */
/* Face geometry                                                             */
/* ------------------------------------------------------------------------ */

typedef struct {
  vec3 p[3];      /* face vertices in frame order */
  vec3 apex;      /* tet vertex opposite the face */
  vec3 e1, e2, n; /* tangent axes and inward unit normal */
  double area;
} face_t;

static void face_of(const double* V, const int32_t* T, int64_t t, int f, face_t* F) {
  const int32_t* tv = T + 4 * t;
  for (int k = 0; k < 3; ++k) F->p[k] = vert(V, tv[(f + 1 + k) % 4]);
  F->apex = vert(V, tv[f]);
  vec3 a = vsub(F->p[1], F->p[0]), b = vsub(F->p[2], F->p[0]);
  vec3 c = vcross(a, b);
  F->area = 0.5 * vnorm(c);
  if (vdot(c, vsub(F->apex, F->p[0])) < 0) c = vscale(c, -1.0);
  F->n = vunit(c);
  F->e1 = ORC_MUTATE == 6 ? a : vunit(a);
  F->e2 = vcross(F->n, F->e1);
}

/* ------------------------------------------------------------------------ */
/* Zernike polynomials (Sec. 3.1): factorial closed form + atan2 angles      */
/* ------------------------------------------------------------------------ */

static double factorial(int k) {
  double r = 1.0;
  for (int i = 2; i <= k; ++i) r *= i;
  return r;
}

/* R_n^m(rho) = sum_k (-1)^k (n-k)! / (k! ((n+m)/2-k)! ((n-m)/2-k)!) rho^(n-2k) */
static double zern_radial(int n, int m, double rho) {
  if (m < 0) m = -m;
  if (m > n || ((n - m) & 1)) return 0.0;
  double s = 0.0;
  for (int k = 0; k <= (n - m) / 2; ++k) {
    double c = factorial(n - k) / (factorial(k) * factorial((n + m) / 2 - k) * factorial((n - m) / 2 - k));
    if (k & 1) c = -c;
    s += c * pow(rho, n - 2 * k);
  }
  return s;
}

static int nbasis(int Np) { return (Np + 1) * (Np + 2) / 2; }

static void zern_all(int Np, double px, double py, double* Z) {
  double rho = sqrt(px * px + py * py);
  double phi = rho > 0.0 ? atan2(py, px) : 0.0;
  for (int n = 0; n <= Np; ++n)
    for (int m = -n; m <= n; m += 2) {
      int idx = (n * (n + 2) + m) / 2;
      double R = zern_radial(n, m, rho);
      Z[idx] = (m >= 0 || ORC_MUTATE == 1) ? R * cos(m * phi) : R * sin(-m * phi);
    }
}

/* inverse norm N_{nm} = (2n+2)/(eps_m pi), eps_0 = 2 */
static double zern_invnorm(int n, int m) {
  return (2.0 * n + 2.0) / ((m == 0 && ORC_MUTATE != 2 ? 2.0 : 1.0) * M_PI);
}

void orc_zernike(int Np, int64_t npts, const double* px, const double* py, double* out) {
  int nb = nbasis(Np);
  for (int64_t i = 0; i < npts; ++i) zern_all(Np, px[i], py[i], out + i * nb);
}

/* ------------------------------------------------------------------------ */
/* Spatial integral S_{l->l'}(d) by projection and clipping (Sec. 3.3)       */
/* ------------------------------------------------------------------------ */

typedef struct { double x, y, L; } pt2;

/* Clip a convex polygon (in face-plane coordinates, carrying the affine value L)
 * against the half-plane a*x + b*y + c >= 0. */
static int clip_half(const pt2* in, int nin, pt2* out, double a, double b, double c) {
  int nout = 0;
  for (int i = 0; i < nin; ++i) {
    pt2 P = in[i], Q = in[(i + 1) % nin];
    double fp = a * P.x + b * P.y + c, fq = a * Q.x + b * Q.y + c;
    if (fp >= 0) out[nout++] = P;
    if ((fp >= 0) != (fq >= 0)) {
      double s = fp / (fp - fq);
      pt2 R = {P.x + s * (Q.x - P.x), P.y + s * (Q.y - P.y), P.L + s * (Q.L - P.L)};
      out[nout++] = R;
    }
  }
  return nout;
}

/* Integral of exp(-mu L) (and of -L exp(-mu L)) over a triangle whose vertex
 * values of the affine function L are given; collapsed (Duffy) tensor Gauss. */
static void tri_exp_integral(pt2 A, pt2 B, pt2 C, double mu, int nq, const double* gx, const double* gw,
                             double* val, double* dval) {
  double area = 0.5 * fabs((B.x - A.x) * (C.y - A.y) - (C.x - A.x) * (B.y - A.y));
  double s = 0.0, ds = 0.0;
  for (int i = 0; i < nq; ++i) {
    double u = 0.5 * (1.0 + gx[i]);
    for (int j = 0; j < nq; ++j) {
      double v = (1.0 - u) * 0.5 * (1.0 + gx[j]);
      double w = gw[i] * gw[j] * 0.25 * (1.0 - u); /* du dv on the unit simplex */
      double L = A.L + u * (B.L - A.L) + v * (C.L - A.L);
      double e = exp(-(ORC_MUTATE == 4 ? 0.5 : 1.0) * mu * L);
      s += w * e;
      ds += w * (-L * e);
    }
  }
  *val += 2.0 * area * s;
  *dval += 2.0 * area * ds;
}

/* S(d) = Int_{s in src, ray s + t d exits through dst} exp(-mu L(s)) ds.
 * dst: the three vertices of the destination face, dst_n its outward unit
 * normal (pointing out of the tet).  Returns also dS/dmu and the clipped area. */
static double spatial_clip(const face_t* src, const vec3* dst, vec3 dst_n, vec3 d, double mu, int nq,
                           const double* gx, const double* gw, double* dS, double* area_out) {
  double dn = vdot(d, src->n);
  double ddst = vdot(d, dst_n);
  pt2 poly[16], tmp[16];
  int np = 3;
  for (int k = 0; k < 3; ++k) {
    /* project dst vertex X onto the source plane along d: X' = X - t d */
    double t = vdot(vsub(dst[k], src->p[0]), src->n) / dn;
    vec3 Xp = vsub(dst[k], vscale(d, t));
    vec3 r = vsub(Xp, src->p[0]);
    poly[k].x = vdot(r, src->e1);
    poly[k].y = vdot(r, src->e2);
    poly[k].L = t; /* distance from X' to X along d */
  }
  (void)ddst;
  /* source triangle in plane coordinates, counter-clockwise */
  double sx[3], sy[3];
  for (int k = 0; k < 3; ++k) {
    vec3 r = vsub(src->p[k], src->p[0]);
    sx[k] = vdot(r, src->e1);
    sy[k] = vdot(r, src->e2);
  }
  double orient = (sx[1] - sx[0]) * (sy[2] - sy[0]) - (sx[2] - sx[0]) * (sy[1] - sy[0]);
  double sgn = orient > 0 ? 1.0 : -1.0;
  /* make the projected destination polygon counter-clockwise too (not needed
   * for clipping correctness, only for the fan) */
  for (int k = 0; k < 3 && np > 0 && ORC_MUTATE != 7; ++k) {
    int k1 = (k + 1) % 3;
    double ex = sx[k1] - sx[k], ey = sy[k1] - sy[k];
    /* inside: sgn * cross(edge, p - start) >= 0 */
    double a = -sgn * ey, b = sgn * ex, c = -(a * sx[k] + b * sy[k]);
    np = clip_half(poly, np, tmp, a, b, c);
    memcpy(poly, tmp, sizeof(pt2) * np);
  }
  double S = 0.0, dSv = 0.0, area = 0.0;
  for (int k = 1; k + 1 < np; ++k) {
    tri_exp_integral(poly[0], poly[k], poly[k + 1], mu, nq, gx, gw, &S, &dSv);
    area += 0.5 * fabs((poly[k].x - poly[0].x) * (poly[k + 1].y - poly[0].y) -
                       (poly[k + 1].x - poly[0].x) * (poly[k].y - poly[0].y));
  }
  if (dS) *dS = dSv;
  if (area_out) *area_out = area;
  return S;
}

/* ------------------------------------------------------------------------ */
/* Linear spatial basis on each face (the higher-order spatial               */
/* approximation the paper suggests in Sec. 3.1 and at the end of Sec. 4.1)  */
/* ------------------------------------------------------------------------ */

/* (1/|T|) Int_T (sum_k u_k l_k)(sum_k v_k l_k) over a triangle in barycentric
 * coordinates l_k: the mass matrix of barycentrics is |T| (1 + delta_ij) / 12. */
static double p1_ip(const double* u, const double* v) {
  return (u[0] * v[0] + u[1] * v[1] + u[2] * v[2] +
          (ORC_MUTATE == 13 ? 0.0 : 1.0) * (u[0] + u[1] + u[2]) * (v[0] + v[1] + v[2])) / 12.0;
}

/* L2-orthonormal basis of the affine functions on a face, by Gram-Schmidt of
 * (1, l_1, l_2) in this order (l_k the barycentric coordinate of the face's
 * k-th vertex in frame order): sqrt|T| phi_a = sum_k C[a][k] l_k. */
static void p1_coeffs(double C[3][3]) {
  const double F[3][3] = {{1.0, 1.0, 1.0}, {0.0, 1.0, 0.0}, {0.0, 0.0, 1.0}};
  for (int a = 0; a < 3; ++a) {
    double v[3] = {F[a][0], F[a][1], F[a][2]};
    for (int c = 0; c < a; ++c) {
      double pr = p1_ip(v, C[c]);
      for (int k = 0; k < 3; ++k) v[k] -= pr * C[c][k];
    }
    double nrm = sqrt(p1_ip(v, v));
    for (int k = 0; k < 3; ++k) C[a][k] = v[k] / nrm;
  }
}

/* the coefficients C[a][k] of p1_coeffs, row-major (for checks) */
void orc_p1_coeffs(double* out) {
  double C[3][3];
  p1_coeffs(C);
  for (int a = 0; a < 3; ++a)
    for (int k = 0; k < 3; ++k) out[3 * a + k] = C[a][k];
}

typedef struct { double x, y, L, b[3]; } pt2b;

static int clip_half_b(const pt2b* in, int nin, pt2b* out, double a, double b, double c) {
  int nout = 0;
  for (int i = 0; i < nin; ++i) {
    pt2b P = in[i], Q = in[(i + 1) % nin];
    double fp = a * P.x + b * P.y + c, fq = a * Q.x + b * Q.y + c;
    if (fp >= 0) out[nout++] = P;
    if ((fp >= 0) != (fq >= 0)) {
      double s = fp / (fp - fq);
      pt2b R;
      R.x = P.x + s * (Q.x - P.x);
      R.y = P.y + s * (Q.y - P.y);
      R.L = P.L + s * (Q.L - P.L);
      for (int k = 0; k < 3; ++k) R.b[k] = P.b[k] + s * (Q.b[k] - P.b[k]);
      out[nout++] = R;
    }
  }
  return nout;
}

/* Linear-basis spatial matrix of direction d:
 *   S[b][a] = Int_{s in src, ray s + t d exits through dst} (sqrt|T_l| phi_a)(s) (sqrt|T_l'| psi_b)(y(s)) exp(-mu L(s)) ds,
 * y(s) = s + L(s) d the exit point on dst, phi the basis of the source face,
 * psi that of the receiving row's face, whose vertex perm[k] is dst->p[k].
 * The projection of dst onto the source plane along d carries the
 * barycentric coordinates of y on dst, clipped together with the polygon
 * (the projection is affine).  dS: d/dmu.  Returns S[0][0]. */
static double spatial_clip_p1(const face_t* src, const face_t* dst, const int* perm, vec3 d, double mu, int nq,
                              const double* gx, const double* gw, const double C[3][3], double* S, double* dS) {
  double dn = vdot(d, src->n);
  pt2b poly[16], tmp[16];
  int np = 3;
  for (int k = 0; k < 3; ++k) {
    double t = vdot(vsub(dst->p[k], src->p[0]), src->n) / dn;
    vec3 r = vsub(vsub(dst->p[k], vscale(d, t)), src->p[0]);
    poly[k].x = vdot(r, src->e1);
    poly[k].y = vdot(r, src->e2);
    poly[k].L = t;
    for (int c = 0; c < 3; ++c) poly[k].b[c] = c == k ? 1.0 : 0.0;
  }
  double sx[3], sy[3];
  for (int k = 0; k < 3; ++k) {
    vec3 r = vsub(src->p[k], src->p[0]);
    sx[k] = vdot(r, src->e1);
    sy[k] = vdot(r, src->e2);
  }
  double orient = (sx[1] - sx[0]) * (sy[2] - sy[0]) - (sx[2] - sx[0]) * (sy[1] - sy[0]);
  double sgn = orient > 0 ? 1.0 : -1.0;
  for (int k = 0; k < 3 && np > 0; ++k) {
    int k1 = (k + 1) % 3;
    double ex = sx[k1] - sx[k], ey = sy[k1] - sy[k];
    double a = -sgn * ey, b = sgn * ex, c = -(a * sx[k] + b * sy[k]);
    np = clip_half_b(poly, np, tmp, a, b, c);
    memcpy(poly, tmp, sizeof(pt2b) * np);
  }
  /* source barycentrics l_1, l_2 of a plane point from the inverse edge matrix */
  double m00 = sx[1] - sx[0], m01 = sx[2] - sx[0], m10 = sy[1] - sy[0], m11 = sy[2] - sy[0];
  double det = m00 * m11 - m01 * m10;
  for (int k = 0; k < 9; ++k) S[k] = dS[k] = 0.0;
  for (int k = 1; k + 1 < np; ++k) {
    const pt2b *A = &poly[0], *B = &poly[k], *Cc = &poly[k + 1];
    double area = 0.5 * fabs((B->x - A->x) * (Cc->y - A->y) - (Cc->x - A->x) * (B->y - A->y));
    for (int i = 0; i < nq; ++i) {
      double u = 0.5 * (1.0 + gx[i]);
      for (int j = 0; j < nq; ++j) {
        double v = (1.0 - u) * 0.5 * (1.0 + gx[j]);
        double w = 2.0 * area * gw[i] * gw[j] * 0.25 * (1.0 - u);
        double x = A->x + u * (B->x - A->x) + v * (Cc->x - A->x);
        double y = A->y + u * (B->y - A->y) + v * (Cc->y - A->y);
        double L = A->L + u * (B->L - A->L) + v * (Cc->L - A->L);
        double ls[3], lr[3];
        ls[1] = (m11 * x - m01 * y) / det;
        ls[2] = (-m10 * x + m00 * y) / det;
        ls[0] = 1.0 - ls[1] - ls[2];
        for (int c = 0; c < 3; ++c)
          lr[perm[c]] = A->b[c] + u * (B->b[c] - A->b[c]) + v * (Cc->b[c] - A->b[c]);
        if (ORC_MUTATE == 12) /* the receiving function read at the source point */
          for (int c = 0; c < 3; ++c) lr[c] = ls[c];
        double ph[3], ps[3];
        for (int a = 0; a < 3; ++a) {
          ph[a] = C[a][0] * ls[0] + C[a][1] * ls[1] + C[a][2] * ls[2];
          ps[a] = C[a][0] * lr[0] + C[a][1] * lr[1] + C[a][2] * lr[2];
        }
        double e = exp(-mu * L);
        for (int bb = 0; bb < 3; ++bb)
          for (int a = 0; a < 3; ++a) {
            S[bb * 3 + a] += w * e * ps[bb] * ph[a];
            dS[bb * 3 + a] += w * (-L * e) * ps[bb] * ph[a];
          }
      }
    }
  }
  return S[0];
}

/* position k' in face g's frame order of the vertex of face f at position k */
static void face_perm(const face_t* f, const face_t* g, int* perm) {
  for (int k = 0; k < 3; ++k) {
    perm[k] = 0;
    for (int k2 = 0; k2 < 3; ++k2)
      if (f->p[k].x == g->p[k2].x && f->p[k].y == g->p[k2].y && f->p[k].z == g->p[k2].z) perm[k] = k2;
  }
}

/* ------------------------------------------------------------------------ */
/* Direction sub-regions (Sec. 3.3-3.4)                                      */
/* ------------------------------------------------------------------------ */

/* For source face l and destination face l' of the same tet: A = the source
 * vertex not on l' (tet vertex l'), B and C the two shared vertices (in face
 * order), D the apex (tet vertex l).  The point P where the ray through D
 * meets the source plane falls in one of seven regions cut out by the lines
 * AB, BC, CA; as directions these are spherical polygons with generators
 *   0 interior      {D-A, D-B, D-C}
 *   1 wedge at A    {D-A, B-A, C-A}
 *   2 strip on AB   {D-A, D-B, C-B, C-A}
 *   3 strip on AC   {D-A, D-C, B-C, B-A}
 *   4 wedge at B    {D-B, C-B, A-B}
 *   5 wedge at C    {D-C, A-C, B-C}
 *   6 strip on BC   {D-B, D-C, A-C, A-B}
 * Regions 4-6 give an empty integration triangle for l' (Sec. 3.3). */
static int region_generators(const face_t* src, vec3 A, vec3 B, vec3 C, int region, vec3* g) {
  vec3 D = src->apex;
  switch (region) {
    case 0: g[0] = vsub(D, A); g[1] = vsub(D, B); g[2] = vsub(D, C); return 3;
    case 1: g[0] = vsub(D, A); g[1] = vsub(B, A); g[2] = vsub(C, A); return 3;
    case 2: g[0] = vsub(D, A); g[1] = vsub(D, B); g[2] = vsub(C, B); g[3] = vsub(C, A); return 4;
    case 3: g[0] = vsub(D, A); g[1] = vsub(D, C); g[2] = vsub(B, C); g[3] = vsub(B, A); return 4;
    case 4: g[0] = vsub(D, B); g[1] = vsub(C, B); g[2] = vsub(A, B); return 3;
    case 5: g[0] = vsub(D, C); g[1] = vsub(A, C); g[2] = vsub(B, C); return 3;
    default: g[0] = vsub(D, B); g[1] = vsub(D, C); g[2] = vsub(A, C); g[3] = vsub(A, B); return 4;
  }
}

/* Bilinear map of Eq. (Parametr) through unit generators v1..v4 (v4 = v1 for a
 * triangle).  Returns the unit direction and the Jacobian of Sec. 3.4, which
 * includes the factor cos(theta) = sin(2 theta)/(2 sin theta). */
static vec3 bilinear_dir(const vec3* v, double xi, double eta, vec3 n, double* jac) {
  vec3 a = vscale(vadd(vadd(v[0], v[1]), vadd(v[2], v[3])), 0.25);
  vec3 b = vscale(vsub(vadd(v[1], v[2]), vadd(v[0], v[3])), 0.25);
  vec3 c = vscale(vsub(vadd(v[2], v[3]), vadd(v[0], v[1])), 0.25);
  vec3 dd = vscale(vsub(vadd(v[2], v[0]), vadd(v[3], v[1])), 0.25);
  vec3 f = vadd(vadd(a, vscale(b, xi)), vadd(vscale(c, eta), vscale(dd, xi * eta)));
  vec3 fx = vadd(b, vscale(dd, eta));
  vec3 fe = vadd(c, vscale(dd, xi));
  double r = vnorm(f);
  double det = vdot(f, vcross(fx, fe));
  *jac = fabs(vdot(f, n) * det) / (r * r * r * r);
  return vscale(f, 1.0 / r);
}

static void region_unit_gens(const face_t* src, vec3 A, vec3 B, vec3 C, int region, vec3* v) {
  vec3 g[4];
  int ng = region_generators(src, A, B, C, region, g);
  for (int k = 0; k < ng; ++k) v[k] = vunit(g[k]);
  if (ng == 3) v[3] = v[0];
}

/* projected solid angle Int cos(theta) dw of one region by the quadrature */
double orc_region_cos_measure(const double* V, const int32_t* T, int64_t t, int f, int fp, int region, int q,
                              const double* gx, const double* gw) {
  face_t src;
  face_of(V, T, t, f, &src);
  const int32_t* tv = T + 4 * t;
  vec3 A = vert(V, tv[fp]);
  vec3 BC[2];
  int nb = 0;
  for (int k = 0; k < 4; ++k)
    if (k != f && k != fp) BC[nb++] = vert(V, tv[k]);
  vec3 v[4];
  region_unit_gens(&src, A, BC[0], BC[1], region, v);
  double s = 0.0;
  for (int i = 0; i < q; ++i)
    for (int j = 0; j < q; ++j) {
      double jac;
      bilinear_dir(v, gx[i], gx[j], src.n, &jac);
      s += gw[i] * gw[j] * jac;
    }
  return s;
}

/* ------------------------------------------------------------------------ */
/* One operator block                                                        */
/* ------------------------------------------------------------------------ */

/* Block for source face (t,f) -> destination face fp of tet t, received by row
 * recv_row (the neighbour's row across fp, or 4t+fp on the boundary), with
 * weight lam and damping mu of tet t.  out: nb x nb row-major, row = test
 * index (n',m') on the receiving face, column = trial index (n,m) on the
 * source face.  dout (optional): d(block)/d(mu).  regions_mask selects which
 * of the seven direction regions are integrated (0x0F = the four non-empty
 * ones; 0x7F = all seven, for checks). */
/* Heterogeneous media at the exit face fp (Sec. 3.3): kind 0 = no interface
 * (constant lambda: transmission with probability 1 in uniform media, or a
 * boundary reflection with weight r); kind 1 = the part transmitted into the
 * neighbour, weight lambda_t(d), received with the tangential direction
 * scaled by c_ratio = c_i / c_j (Snell's law, sin(theta_t) = (c_i/c_j)
 * sin(theta_r)); kind 2 = the part reflected back into tet t, weight
 * 1 - lambda_t(d), received on face (t, fp) itself with the specularly
 * reflected direction (same tangential components).  z_src = z_j, z_dst = z_i
 * are the impedances rho_f c of the two tets. */
typedef struct {
  int kind;
  double c_ratio, z_src, z_dst;
} media_t;

/* lambda_t = 4 z_i z_j cos(theta_r) cos(theta_t) / (z_i cos(theta_r) + z_j cos(theta_t))^2,
 * zero beyond the critical angle (total internal reflection) */
static double transmission(double cos_r, double c_ratio, double z_src, double z_dst) {
  double s2 = c_ratio * c_ratio * (1.0 - cos_r * cos_r);
  if (s2 >= 1.0) return 0.0;
  double cos_t = sqrt(1.0 - s2);
  double den = ORC_MUTATE == 9 ? z_src * cos_r + z_dst * cos_t : z_dst * cos_r + z_src * cos_t;
  return 4.0 * z_dst * z_src * cos_r * cos_t / (den * den);
}

double orc_transmission(double cos_r, double c_ratio, double z_src, double z_dst) {
  return transmission(cos_r, c_ratio, z_src, z_dst);
}

static void block_fixed(const double* V, const int32_t* T, int64_t t, int f, int fp, int64_t recv_row,
                        double mu, double lam, int Np, int q, const double* gx, const double* gw, int nq_tri,
                        const double* tx, const double* tw, int regions_mask, const media_t* md, int ns,
                        double* out, double* dout) {
  int nb = nbasis(Np);
  int nbe = ns * nb; /* ns spatial functions per face (1: constant, 3: linear), index s nb + idx */
  face_t src, dstf, recv;
  face_of(V, T, t, f, &src);
  face_of(V, T, t, fp, &dstf);
  face_of(V, T, recv_row / 4, (int)(recv_row % 4), &recv);
  double Cp1[3][3];
  int perm[3] = {0, 1, 2};
  if (ns == 3) {
    p1_coeffs(Cp1);
    face_perm(&dstf, &recv, perm);
  }
  const int kind = md ? md->kind : 0;
  const double c_ratio = kind == 1 ? md->c_ratio : 1.0;
  const int32_t* tv = T + 4 * t;
  vec3 A = vert(V, tv[fp]);
  vec3 BC[2];
  int k2 = 0;
  for (int k = 0; k < 4; ++k)
    if (k != f && k != fp) BC[k2++] = vert(V, tv[k]);
  vec3 dst_n_out = vscale(dstf.n, -1.0);
  double* Zp = (double*)malloc(sizeof(double) * nb);
  double* Zq = (double*)malloc(sizeof(double) * nb);
  memset(out, 0, sizeof(double) * nbe * nbe);
  if (dout) memset(dout, 0, sizeof(double) * nbe * nbe);
  for (int region = 0; region < 7; ++region) {
    if (!(regions_mask & (1 << region))) continue;
    vec3 v[4];
    region_unit_gens(&src, A, BC[0], BC[1], region, v);
    for (int i = 0; i < q; ++i)
      for (int j = 0; j < q; ++j) {
        double jac;
        vec3 d = bilinear_dir(v, gx[i], gx[j], src.n, &jac);
        double w = gw[i] * gw[j] * jac;
        double dS;
        double Sm[9], dSm[9];
        double S;
        if (ns == 1) {
          S = spatial_clip(&src, dstf.p, dst_n_out, d, mu, nq_tri, tx, tw, &dS, NULL);
        } else {
          S = spatial_clip_p1(&src, &dstf, perm, d, mu, nq_tri, tx, tw, (const double(*)[3])Cp1, Sm, dSm);
          dS = dSm[0];
        }
        if (S == 0.0 && dS == 0.0) continue;
        if (kind) {
          double lt = transmission(-vdot(d, dstf.n), md->c_ratio, md->z_src, md->z_dst);
          double wl = kind == 1 ? lt : (ORC_MUTATE == 11 ? lt : 1.0 - lt);
          if (wl == 0.0) continue;
          w *= wl;
        }
        zern_all(Np, vdot(d, src.e1), vdot(d, src.e2), Zp);
        if (ORC_MUTATE == 3)
          zern_all(Np, vdot(d, src.e1), vdot(d, src.e2), Zq);
        else
          zern_all(Np, (ORC_MUTATE == 10 && kind == 1 ? 1.0 / c_ratio : c_ratio) * vdot(d, recv.e1),
                   (ORC_MUTATE == 10 && kind == 1 ? 1.0 / c_ratio : c_ratio) * vdot(d, recv.e2), Zq);
        if (ns == 1) {
          for (int a = 0; a < nb; ++a) {
            double wa = w * Zq[a];
            for (int b = 0; b < nb; ++b) {
              out[a * nb + b] += wa * S * Zp[b];
              if (dout) dout[a * nb + b] += wa * dS * Zp[b];
            }
          }
        } else {
          /* row (sb, a): test spatial function sb, Zernike a; column (sa, b) */
          for (int sb = 0; sb < 3; ++sb)
            for (int a = 0; a < nb; ++a) {
              double wa = w * Zq[a];
              double* orow = out + (int64_t)(sb * nb + a) * nbe;
              double* drow = dout ? dout + (int64_t)(sb * nb + a) * nbe : NULL;
              for (int sa = 0; sa < 3; ++sa) {
                double v = wa * Sm[sb * 3 + sa], dv = wa * dSm[sb * 3 + sa];
                for (int b = 0; b < nb; ++b) {
                  orow[sa * nb + b] += v * Zp[b];
                  if (drow) drow[sa * nb + b] += dv * Zp[b];
                }
              }
            }
        }
      }
  }
  double sc = lam / sqrt(src.area * dstf.area);
  for (int sb = 0; sb < ns; ++sb)
    for (int n = 0; n <= Np; ++n)
      for (int m = -n; m <= n; m += 2) {
        int a = sb * nb + (n * (n + 2) + m) / 2;
        double s = sc * zern_invnorm(n, m);
        for (int b = 0; b < nbe; ++b) {
          out[a * nbe + b] *= s;
          if (dout) dout[a * nbe + b] *= s;
        }
      }
  free(Zp);
  free(Zq);
}

/* Gauss-Legendre table: levels k = 0..nlev-1 with orders qs[k], nodes/weights
 * at offset offs[k] in gx/gw. */
typedef struct {
  int nlev;
  const int* qs;
  const int* offs;
  const double* gx;
  const double* gw;
} gl_table;

/* Blocks for a list of face pairs.  Fixed order: level = lev0 only (rtol <= 0).
 * Adaptive: start at level lev0, double (next level) until the block max-norm
 * change is <= rtol * block max-norm; q_used returns the accepted order (or
 * -order if the top level was reached without meeting rtol). */
static int blocks_adaptive(const double* V, const int32_t* T, int64_t npairs, const int64_t* tet,
                           const int32_t* f, const int32_t* fp, const int64_t* recv_row, const double* mu,
                           const double* lam, const int32_t* kind, const double* c_ratio, const double* z_src,
                           const double* z_dst, int Np, int nlev, const int* qs, const int* offs,
                           const double* gx, const double* gw, int lev0, double rtol, int tri_lev,
                           int regions_mask, int ns, int nthreads, double* out, double* dout, int32_t* q_used) {
  int nb = ns * nbasis(Np); /* block side with ns spatial functions per face */
  gl_table G = {nlev, qs, offs, gx, gw};
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
#pragma omp parallel
  {
    double* prev = (double*)malloc(sizeof(double) * nb * nb);
    double* prevd = (double*)malloc(sizeof(double) * nb * nb);
#pragma omp for schedule(dynamic, 4)
    for (int64_t i = 0; i < npairs; ++i) {
      double* o = out + i * nb * nb;
      double* od = dout ? dout + i * nb * nb : NULL;
      const double* tx = G.gx + G.offs[tri_lev];
      const double* tw = G.gw + G.offs[tri_lev];
      int nt = G.qs[tri_lev];
      int lev = lev0;
      media_t mdi;
      const media_t* md = NULL;
      if (kind) {
        mdi.kind = kind[i];
        mdi.c_ratio = c_ratio[i];
        mdi.z_src = z_src[i];
        mdi.z_dst = z_dst[i];
        md = &mdi;
      }
      block_fixed(V, T, tet[i], f[i], fp[i], recv_row[i], mu[i], lam[i], Np, G.qs[lev], G.gx + G.offs[lev],
                  G.gw + G.offs[lev], nt, tx, tw, regions_mask, md, ns, o, od);
      int accepted = rtol > 0 ? -G.qs[lev] : G.qs[lev];
      while (rtol > 0 && lev + 1 < G.nlev) {
        memcpy(prev, o, sizeof(double) * nb * nb);
        if (od) memcpy(prevd, od, sizeof(double) * nb * nb);
        ++lev;
        block_fixed(V, T, tet[i], f[i], fp[i], recv_row[i], mu[i], lam[i], Np, G.qs[lev], G.gx + G.offs[lev],
                    G.gw + G.offs[lev], nt, tx, tw, regions_mask, md, ns, o, od);
        double dmax = 0.0, bmax = 0.0, ddmax = 0.0, dbmax = 0.0;
        for (int k = 0; k < nb * nb; ++k) {
          dmax = fmax(dmax, fabs(o[k] - prev[k]));
          bmax = fmax(bmax, fabs(o[k]));
          if (od) {
            ddmax = fmax(ddmax, fabs(od[k] - prevd[k]));
            dbmax = fmax(dbmax, fabs(od[k]));
          }
        }
        if (dmax <= rtol * bmax && (!od || ddmax <= rtol * dbmax)) {
          accepted = G.qs[lev];
          break;
        }
        accepted = -G.qs[lev];
      }
      if (q_used) q_used[i] = accepted;
    }
    free(prev);
    free(prevd);
  }
  return 0;
}

int orc_blocks(const double* V, const int32_t* T, int64_t npairs, const int64_t* tet, const int32_t* f,
               const int32_t* fp, const int64_t* recv_row, const double* mu, const double* lam, int Np,
               int nlev, const int* qs, const int* offs, const double* gx, const double* gw, int lev0,
               double rtol, int tri_lev, int regions_mask, int nthreads, double* out, double* dout,
               int32_t* q_used) {
  return blocks_adaptive(V, T, npairs, tet, f, fp, recv_row, mu, lam, NULL, NULL, NULL, NULL, Np, nlev, qs, offs,
                         gx, gw, lev0, rtol, tri_lev, regions_mask, 1, nthreads, out, dout, q_used);
}

/* As orc_blocks with the linear spatial basis (3 functions per face): blocks
 * of side 3 nb, index s nb + idx for spatial function s and Zernike idx. */
int orc_blocks_p1(const double* V, const int32_t* T, int64_t npairs, const int64_t* tet, const int32_t* f,
                  const int32_t* fp, const int64_t* recv_row, const double* mu, const double* lam, int Np, int nlev,
                  const int* qs, const int* offs, const double* gx, const double* gw, int lev0, double rtol,
                  int tri_lev, int regions_mask, int nthreads, double* out, double* dout, int32_t* q_used) {
  return blocks_adaptive(V, T, npairs, tet, f, fp, recv_row, mu, lam, NULL, NULL, NULL, NULL, Np, nlev, qs, offs,
                         gx, gw, lev0, rtol, tri_lev, regions_mask, 3, nthreads, out, dout, q_used);
}

/* As orc_blocks, with per-pair media (kind, c_ratio, z_src, z_dst; see media_t). */
int orc_blocks_media(const double* V, const int32_t* T, int64_t npairs, const int64_t* tet, const int32_t* f,
                     const int32_t* fp, const int64_t* recv_row, const double* mu, const double* lam,
                     const int32_t* kind, const double* c_ratio, const double* z_src, const double* z_dst, int Np,
                     int nlev, const int* qs, const int* offs, const double* gx, const double* gw, int lev0,
                     double rtol, int tri_lev, int regions_mask, int nthreads, double* out, double* dout,
                     int32_t* q_used) {
  return blocks_adaptive(V, T, npairs, tet, f, fp, recv_row, mu, lam, kind, c_ratio, z_src, z_dst, Np, nlev, qs,
                         offs, gx, gw, lev0, rtol, tri_lev, regions_mask, 1, nthreads, out, dout, q_used);
}

/* ------------------------------------------------------------------------ */
/* Monte Carlo ray tracing of one block (brute-force pin)                   */
/* ------------------------------------------------------------------------ */

static uint64_t splitmix64(uint64_t* s) {
  uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
static double urand(uint64_t* s) { return (splitmix64(s) >> 11) * (1.0 / 9007199254740992.0); }

/* Estimate of the block (t,f)->(t,fp) received by recv_row, and its standard
 * error, from nsamp samples: s uniform on face f, p uniform on the unit disc
 * (a cosine-weighted inward direction), the ray traced to the face it leaves
 * through; B = lam N_{n'm'} pi sqrt(A_l/A_l') E[Z(p') Z(p) exp(-mu L) 1{exit=l'}]. */
static int mc_block(const double* V, const int32_t* T, int64_t t, int f, int fp, int64_t recv_row, double mu,
                    double lam, const media_t* md, int Np, int ns, int64_t nsamp, uint64_t seed, int nthreads,
                    double* mean, double* stderr_) {
  int nz = nbasis(Np);
  int nb = ns * nz; /* block side; with ns = 3 the score carries phi_a(s) psi_b(exit point) */
  const int kind = md ? md->kind : 0;
  const double c_ratio = kind == 1 ? md->c_ratio : 1.0;
  face_t src, recv, faces[4];
  face_of(V, T, t, f, &src);
  face_of(V, T, recv_row / 4, (int)(recv_row % 4), &recv);
  for (int k = 0; k < 4; ++k) face_of(V, T, t, k, &faces[k]);
  double Cp1[3][3];
  p1_coeffs(Cp1);
  /* receiving face: plane coordinates of its vertices for barycentrics */
  double rx[3], ry[3];
  for (int k = 0; k < 3; ++k) {
    vec3 r = vsub(recv.p[k], recv.p[0]);
    rx[k] = vdot(r, recv.e1);
    ry[k] = vdot(r, recv.e2);
  }
  const double rdet = (rx[1] - rx[0]) * (ry[2] - ry[0]) - (rx[2] - rx[0]) * (ry[1] - ry[0]);
  double* S1 = (double*)calloc(nb * nb, sizeof(double));
  double* S2 = (double*)calloc(nb * nb, sizeof(double));
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
#pragma omp parallel
  {
    double* s1 = (double*)calloc(nb * nb, sizeof(double));
    double* s2 = (double*)calloc(nb * nb, sizeof(double));
    double* Zp = (double*)malloc(sizeof(double) * nb);
    double* Zq = (double*)malloc(sizeof(double) * nb);
    double ph[3] = {1.0, 0.0, 0.0}, ps[3] = {1.0, 0.0, 0.0};
#pragma omp for schedule(static)
    for (int64_t chunk = 0; chunk < 1024; ++chunk) {
      /* independent stream per chunk: start at a hashed point of the 2^64 cycle */
      uint64_t h = seed ^ ((uint64_t)chunk * 0xD1B54A32D192ED03ull);
      uint64_t st = splitmix64(&h);
      st ^= splitmix64(&h) << 1;
      int64_t lo = nsamp * chunk / 1024, hi = nsamp * (chunk + 1) / 1024;
      for (int64_t i = lo; i < hi; ++i) {
        /* uniform point on the source triangle */
        double r1 = urand(&st), r2 = urand(&st);
        if (r1 + r2 > 1.0) { r1 = 1.0 - r1; r2 = 1.0 - r2; }
        vec3 s = vadd(src.p[0], vadd(vscale(vsub(src.p[1], src.p[0]), r1), vscale(vsub(src.p[2], src.p[0]), r2)));
        /* uniform point on the unit disc by rejection */
        double px, py;
        do {
          px = 2.0 * urand(&st) - 1.0;
          py = 2.0 * urand(&st) - 1.0;
        } while (px * px + py * py >= 1.0);
        double pz = sqrt(1.0 - px * px - py * py);
        vec3 d = vadd(vadd(vscale(src.e1, px), vscale(src.e2, py)), vscale(src.n, pz));
        /* exit face: smallest positive distance to the other three face planes */
        int ex = -1;
        double L = 1e300;
        for (int k = 0; k < 4; ++k) {
          if (k == f) continue;
          double dn = -vdot(d, faces[k].n); /* outward normal component */
          if (dn <= 0) continue;
          double tk = vdot(vsub(s, faces[k].p[0]), faces[k].n) / dn;
          if (tk < L) { L = tk; ex = k; }
        }
        if (ex != fp) continue;
        double e = exp(-mu * L);
        if (kind) {
          double lt = transmission(-vdot(d, faces[fp].n), md->c_ratio, md->z_src, md->z_dst);
          e *= kind == 1 ? lt : 1.0 - lt;
        }
        zern_all(Np, px, py, Zp);
        zern_all(Np, c_ratio * vdot(d, recv.e1), c_ratio * vdot(d, recv.e2), Zq);
        if (ns == 3) {
          /* source point barycentrics (1 - r1 - r2, r1, r2); exit point on the receiving face */
          double ls[3] = {1.0 - r1 - r2, r1, r2}, lr[3];
          vec3 y = vsub(vadd(s, vscale(d, L)), recv.p[0]);
          double yx = vdot(y, recv.e1), yy = vdot(y, recv.e2);
          lr[1] = (yx * (ry[2] - ry[0]) - (rx[2] - rx[0]) * yy) / rdet;
          lr[2] = ((rx[1] - rx[0]) * yy - yx * (ry[1] - ry[0])) / rdet;
          lr[0] = 1.0 - lr[1] - lr[2];
          for (int a = 0; a < 3; ++a) {
            ph[a] = Cp1[a][0] * ls[0] + Cp1[a][1] * ls[1] + Cp1[a][2] * ls[2];
            ps[a] = Cp1[a][0] * lr[0] + Cp1[a][1] * lr[1] + Cp1[a][2] * lr[2];
          }
        }
        for (int sb = 0; sb < ns; ++sb)
          for (int a = 0; a < nz; ++a)
            for (int sa = 0; sa < ns; ++sa)
              for (int b = 0; b < nz; ++b) {
                double x = Zq[a] * Zp[b] * e * ps[sb] * ph[sa];
                int k = (sb * nz + a) * nb + sa * nz + b;
                s1[k] += x;
                s2[k] += x * x;
              }
      }
    }
#pragma omp critical
    for (int k = 0; k < nb * nb; ++k) {
      S1[k] += s1[k];
      S2[k] += s2[k];
    }
    free(s1); free(s2); free(Zp); free(Zq);
  }
  double Adst = faces[fp].area;
  for (int sb = 0; sb < ns; ++sb)
  for (int n = 0; n <= Np; ++n)
    for (int m = -n; m <= n; m += 2) {
      int a = sb * nz + (n * (n + 2) + m) / 2;
      double sc = lam * zern_invnorm(n, m) * M_PI * sqrt(src.area / Adst);
      for (int b = 0; b < nb; ++b) {
        double m1 = S1[a * nb + b] / (double)nsamp;
        double var = S2[a * nb + b] / (double)nsamp - m1 * m1;
        mean[a * nb + b] = sc * m1;
        stderr_[a * nb + b] = fabs(sc) * sqrt(fmax(var, 0.0) / (double)nsamp);
      }
    }
  free(S1);
  free(S2);
  return 0;
}

int orc_mc_block(const double* V, const int32_t* T, int64_t t, int f, int fp, int64_t recv_row, double mu,
                 double lam, int Np, int64_t nsamp, uint64_t seed, int nthreads, double* mean, double* stderr_) {
  return mc_block(V, T, t, f, fp, recv_row, mu, lam, NULL, Np, 1, nsamp, seed, nthreads, mean, stderr_);
}
/* As orc_mc_block with the linear spatial basis: mean, stderr_ [3 nb][3 nb]. */
int orc_mc_block_p1(const double* V, const int32_t* T, int64_t t, int f, int fp, int64_t recv_row, double mu,
                    double lam, int Np, int64_t nsamp, uint64_t seed, int nthreads, double* mean, double* stderr_) {
  return mc_block(V, T, t, f, fp, recv_row, mu, lam, NULL, Np, 3, nsamp, seed, nthreads, mean, stderr_);
}

/* As orc_mc_block, with the media of the exit face (see media_t): the traced
 * ray is weighted by lambda_t(d) (kind 1) or 1 - lambda_t(d) (kind 2). */
int orc_mc_block_media(const double* V, const int32_t* T, int64_t t, int f, int fp, int64_t recv_row, double mu,
                       int kind, double c_ratio, double z_src, double z_dst, int Np, int64_t nsamp, uint64_t seed,
                       int nthreads, double* mean, double* stderr_) {
  media_t md = {kind, c_ratio, z_src, z_dst};
  return mc_block(V, T, t, f, fp, recv_row, mu, 1.0, &md, Np, 1, nsamp, seed, nthreads, mean, stderr_);
}

/* ------------------------------------------------------------------------ */
/* Per-direction spatial quantities (for checks)                            */
/* ------------------------------------------------------------------------ */

/* For direction d (global, need not be unit) from source face (t,f): the clipped
 * area and damped integral for each destination fp != f, plus the brute-force
 * check quantity Int_{face} exp(-mu L_exit) over a grid of nsub^2 sub-triangles
 * is left to callers.  out_S[3], out_area[3] ordered by fp ascending. */
void orc_spatial(const double* V, const int32_t* T, int64_t t, int f, const double* dir, double mu, int nq,
                 const double* gx, const double* gw, double* out_S, double* out_dS, double* out_area) {
  face_t src, dstf;
  face_of(V, T, t, f, &src);
  vec3 d = vunit(v3(dir[0], dir[1], dir[2]));
  int k = 0;
  for (int fp = 0; fp < 4; ++fp) {
    if (fp == f) continue;
    face_of(V, T, t, fp, &dstf);
    out_S[k] = spatial_clip(&src, dstf.p, vscale(dstf.n, -1.0), d, mu, nq, gx, gw, &out_dS[k], &out_area[k]);
    ++k;
  }
}

/* The linear-basis spatial matrix S[b][a] of spatial_clip_p1 for the pair
 * (t, f) -> (t, fp) received by recv_row, direction dir (unit after
 * normalisation), for checks. */
void orc_spatial_p1(const double* V, const int32_t* T, int64_t t, int f, int fp, int64_t recv_row,
                    const double* dir, double mu, int nq, const double* gx, const double* gw, double* out,
                    double* dout) {
  face_t src, dstf, recv;
  face_of(V, T, t, f, &src);
  face_of(V, T, t, fp, &dstf);
  face_of(V, T, recv_row / 4, (int)(recv_row % 4), &recv);
  double C[3][3];
  int perm[3];
  p1_coeffs(C);
  face_perm(&dstf, &recv, perm);
  spatial_clip_p1(&src, &dstf, perm, vunit(v3(dir[0], dir[1], dir[2])), mu, nq, gx, gw, (const double(*)[3])C, out,
                  dout);
}

/* ------------------------------------------------------------------------ */
/* Interior density functional (Sec. 4.1, Eq. IntDens)                      */
/* ------------------------------------------------------------------------ */

/* g-vector of the interior density at point r inside tet t:
 *   rho_T(r) = sum_{l, nm} rho_(t,l,nm) g_(l,nm),
 *   g_(l,nm) = (1/sqrt|T_l|) Int_{T_l} Z_nm(p(s->r)) cos(vartheta) exp(-mu|r-s|)/|r-s|^2 ds
 * (c = 1), with p(s->r) the tangential part of unit(r - s) in face l's frame.
 * out: [4][nb]; dout: d/dmu of the same.  Collapsed Gauss of order nq per face. */
static void interior_g_ns(const double* V, const int32_t* T, int64_t t, const double* r, double mu, int Np,
                          int ns, int nq, const double* gx, const double* gw, double* out, double* dout);

void orc_interior_g(const double* V, const int32_t* T, int64_t t, const double* r, double mu, int Np, int nq,
                    const double* gx, const double* gw, double* out, double* dout) {
  interior_g_ns(V, T, t, r, mu, Np, 1, nq, gx, gw, out, dout);
}

/* The same with the linear spatial basis: out, dout [4][3][nb], the face
 * integrand weighted by sqrt|T_l| phi_s(point) for s = 0, 1, 2. */
void orc_interior_g_p1(const double* V, const int32_t* T, int64_t t, const double* r, double mu, int Np, int nq,
                       const double* gx, const double* gw, double* out, double* dout) {
  interior_g_ns(V, T, t, r, mu, Np, 3, nq, gx, gw, out, dout);
}

static void interior_g_ns(const double* V, const int32_t* T, int64_t t, const double* r, double mu, int Np,
                          int ns, int nq, const double* gx, const double* gw, double* out, double* dout) {
  int nz = nbasis(Np);
  int nb = ns * nz;
  double Cp1[3][3];
  p1_coeffs(Cp1);
  double* Z = (double*)malloc(sizeof(double) * nb);
  vec3 R = v3(r[0], r[1], r[2]);
  for (int l = 0; l < 4; ++l) {
    face_t F;
    face_of(V, T, t, l, &F);
    double* o = out + l * nb;
    double* od = dout + l * nb;
    for (int k = 0; k < nb; ++k) o[k] = od[k] = 0.0;
    vec3 e1 = vsub(F.p[1], F.p[0]), e2 = vsub(F.p[2], F.p[0]);
    for (int i = 0; i < nq; ++i) {
      double u = 0.5 * (1.0 + gx[i]);
      for (int j = 0; j < nq; ++j) {
        double v = (1.0 - u) * 0.5 * (1.0 + gx[j]);
        double w = gw[i] * gw[j] * 0.25 * (1.0 - u) * 2.0 * F.area;
        vec3 s = vadd(F.p[0], vadd(vscale(e1, u), vscale(e2, v)));
        vec3 rs = vsub(R, s);
        double dist = vnorm(rs);
        vec3 dd = vscale(rs, 1.0 / dist);
        double cosv = vdot(dd, F.n);
        double ker = (ORC_MUTATE == 8 ? 1.0 : cosv) * exp(-mu * dist) / (dist * dist);
        zern_all(Np, vdot(dd, F.e1), vdot(dd, F.e2), Z);
        double lb[3] = {1.0 - u - v, u, v};
        for (int sp = 0; sp < ns; ++sp) {
          double ph = ns == 1 ? 1.0 : Cp1[sp][0] * lb[0] + Cp1[sp][1] * lb[1] + Cp1[sp][2] * lb[2];
          for (int k = 0; k < nz; ++k) {
            o[sp * nz + k] += w * ker * ph * Z[k];
            od[sp * nz + k] += w * (-dist) * ker * ph * Z[k];
          }
        }
      }
    }
    double sc = 1.0 / sqrt(F.area);
    for (int k = 0; k < nb; ++k) {
      o[k] *= sc;
      od[k] *= sc;
    }
  }
  free(Z);
}

/* Adaptive version of the same face integral.  A tet's centroid can sit
 * close to one of its faces (thin tets of a jittered mesh); the kernel
 * cos / R^2 then peaks sharply at the foot of r on that face and a fixed
 * tensor rule loses digits.  Here each face triangle is refined 4-way
 * wherever an 8 x 8 collapsed Gauss rule on a triangle and the sum of the same
 * rule on its four children differ by more than tol (absolute, from rtol times
 * the whole-face estimate); leaves contribute their children's sum. */
typedef struct {
  vec3 R;
  double mu;
  int Np, nb, nq;
  const face_t* F;
  const double *gx, *gw;
  double* Z;
  int ns, nz;         /* spatial functions per face (1 or 3), Zernike functions: nb = ns nz */
  double C[3][3];     /* linear basis coefficients (p1_coeffs) */
  double fx[3], fy[3]; /* face vertices in the face's plane coordinates */
} ig_ctx;

/* face barycentrics of a point of face c->F */
static void ig_bary(const ig_ctx* c, vec3 s, double* lb) {
  vec3 r = vsub(s, c->F->p[0]);
  double x = vdot(r, c->F->e1), y = vdot(r, c->F->e2);
  double a = c->fx[1] - c->fx[0], b = c->fx[2] - c->fx[0], cc = c->fy[1] - c->fy[0], d = c->fy[2] - c->fy[0];
  double det = a * d - b * cc;
  lb[1] = (d * x - b * y) / det;
  lb[2] = (-cc * x + a * y) / det;
  lb[0] = 1.0 - lb[1] - lb[2];
}

static void ig_rule(const ig_ctx* c, vec3 A, vec3 B, vec3 C, double* o, double* od) {
  vec3 e1 = vsub(B, A), e2 = vsub(C, A);
  double area = 0.5 * vnorm(vcross(e1, e2));
  for (int k = 0; k < c->nb; ++k) o[k] = od[k] = 0.0;
  for (int i = 0; i < c->nq; ++i) {
    double u = 0.5 * (1.0 + c->gx[i]);
    for (int j = 0; j < c->nq; ++j) {
      double v = (1.0 - u) * 0.5 * (1.0 + c->gx[j]);
      double w = c->gw[i] * c->gw[j] * 0.25 * (1.0 - u) * 2.0 * area;
      vec3 s = vadd(A, vadd(vscale(e1, u), vscale(e2, v)));
      vec3 rs = vsub(c->R, s);
      double dist = vnorm(rs);
      vec3 dd = vscale(rs, 1.0 / dist);
      double ker = (ORC_MUTATE == 8 ? 1.0 : vdot(dd, c->F->n)) * exp(-c->mu * dist) / (dist * dist);
      zern_all(c->Np, vdot(dd, c->F->e1), vdot(dd, c->F->e2), c->Z);
      double lb[3] = {1.0, 0.0, 0.0};
      if (c->ns == 3) ig_bary(c, s, lb);
      for (int sp = 0; sp < c->ns; ++sp) {
        double ph = c->ns == 1 ? 1.0 : c->C[sp][0] * lb[0] + c->C[sp][1] * lb[1] + c->C[sp][2] * lb[2];
        for (int k = 0; k < c->nz; ++k) {
          o[sp * c->nz + k] += w * ker * ph * c->Z[k];
          od[sp * c->nz + k] += w * (-dist) * ker * ph * c->Z[k];
        }
      }
    }
  }
}

static void ig_adapt(const ig_ctx* c, vec3 A, vec3 B, vec3 C, const double* coarse, double tol, int depth,
                     double* out, double* dout) {
  int nb = c->nb;
  vec3 mab = vscale(vadd(A, B), 0.5), mbc = vscale(vadd(B, C), 0.5), mca = vscale(vadd(C, A), 0.5);
  vec3 kids[4][3] = {{A, mab, mca}, {mab, B, mbc}, {mca, mbc, C}, {mab, mbc, mca}};
  double* buf = (double*)malloc(sizeof(double) * 8 * nb);
  double *fine = buf, *dfine = buf + nb;
  for (int k = 0; k < nb; ++k) fine[k] = dfine[k] = 0.0;
  for (int q = 0; q < 4; ++q) {
    double* o = buf + (2 + q) * nb;
    double* od = buf + 6 * nb;
    ig_rule(c, kids[q][0], kids[q][1], kids[q][2], o, od);
    for (int k = 0; k < nb; ++k) {
      fine[k] += o[k];
      dfine[k] += od[k];
    }
  }
  double err = 0.0;
  for (int k = 0; k < nb; ++k) err = fmax(err, fabs(fine[k] - coarse[k]));
  if (err <= tol || depth >= 24) {
    for (int k = 0; k < nb; ++k) {
      out[k] += fine[k];
      dout[k] += dfine[k];
    }
  } else {
    /* the children's own estimates serve as their coarse values */
    double* kid = (double*)malloc(sizeof(double) * 2 * nb);
    for (int q = 0; q < 4; ++q) {
      ig_rule(c, kids[q][0], kids[q][1], kids[q][2], kid, kid + nb);
      ig_adapt(c, kids[q][0], kids[q][1], kids[q][2], kid, tol / 2.0, depth + 1, out, dout);
    }
    free(kid);
  }
  free(buf);
}

/* rho_T functional of tet t at point r with adaptive cubature (relative
 * tolerance rtol per face); layout as orc_interior_g. */
static void interior_g_adaptive_ns(const double* V, const int32_t* T, int64_t t, const double* r, double mu,
                                   int Np, int ns, double rtol, int nq, const double* gx, const double* gw,
                                   double* out, double* dout);

void orc_interior_g_adaptive(const double* V, const int32_t* T, int64_t t, const double* r, double mu, int Np,
                             double rtol, int nq, const double* gx, const double* gw, double* out, double* dout) {
  interior_g_adaptive_ns(V, T, t, r, mu, Np, 1, rtol, nq, gx, gw, out, dout);
}

/* The same with the linear spatial basis: out, dout [4][3][nb]. */
void orc_interior_g_adaptive_p1(const double* V, const int32_t* T, int64_t t, const double* r, double mu, int Np,
                                double rtol, int nq, const double* gx, const double* gw, double* out,
                                double* dout) {
  interior_g_adaptive_ns(V, T, t, r, mu, Np, 3, rtol, nq, gx, gw, out, dout);
}

static void interior_g_adaptive_ns(const double* V, const int32_t* T, int64_t t, const double* r, double mu,
                                   int Np, int ns, double rtol, int nq, const double* gx, const double* gw,
                                   double* out, double* dout) {
  int nb = ns * nbasis(Np);
  double* Z = (double*)malloc(sizeof(double) * nb);
  double* coarse = (double*)malloc(sizeof(double) * 2 * nb);
  for (int l = 0; l < 4; ++l) {
    face_t F;
    face_of(V, T, t, l, &F);
    ig_ctx c = {v3(r[0], r[1], r[2]), mu, Np, nb, nq, &F, gx, gw, Z};
    c.ns = ns;
    c.nz = nbasis(Np);
    p1_coeffs(c.C);
    for (int k = 0; k < 3; ++k) {
      vec3 q = vsub(F.p[k], F.p[0]);
      c.fx[k] = vdot(q, F.e1);
      c.fy[k] = vdot(q, F.e2);
    }
    double* o = out + l * nb;
    double* od = dout + l * nb;
    for (int k = 0; k < nb; ++k) o[k] = od[k] = 0.0;
    ig_rule(&c, F.p[0], F.p[1], F.p[2], coarse, coarse + nb);
    double scale = 0.0;
    for (int k = 0; k < nb; ++k) scale = fmax(scale, fabs(coarse[k]));
    ig_adapt(&c, F.p[0], F.p[1], F.p[2], coarse, rtol * scale, 0, o, od);
    double sc = 1.0 / sqrt(F.area);
    for (int k = 0; k < nb; ++k) {
      o[k] *= sc;
      od[k] *= sc;
    }
  }
  free(coarse);
  free(Z);
}

/* Adaptive functional of every tet at its centroid, in parallel over tets:
 * out, dout [nt][4][nb]. */
void orc_centroid_g_adaptive(const double* V, const int32_t* T, int64_t nt, const double* mu_tet, int Np, double rtol,
                             int nq, const double* gx, const double* gw, int nthreads, double* out, double* dout) {
  int nb = nbasis(Np);
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t t = 0; t < nt; ++t) {
    double r[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < 4; ++k)
      for (int d = 0; d < 3; ++d) r[d] += 0.25 * V[3 * (int64_t)T[4 * t + k] + d];
    orc_interior_g_adaptive(V, T, t, r, mu_tet[t], Np, rtol, nq, gx, gw, out + t * 4 * nb, dout + t * 4 * nb);
  }
}

/* ------------------------------------------------------------------------ */
/* FP64 operator application in the oracle's own layout                      */
/* ------------------------------------------------------------------------ */

/* Oracle layout: column J = 4t+f owns 3 blocks (destination faces fp != f in
 * ascending order), blocks[J][k][nb][nb], received by dest[J][k].
 * y = x0 + alpha * B x  (trans = 0) or  y = x0 + alpha * B^T x  (trans = 1).
 * x, y, x0: [nrows][nb] for a single right-hand side. */
void orc_apply(int64_t nrows, int nb, const double* blocks, const int64_t* dest, const double* x,
               const double* x0, double alpha, int trans, int nthreads, double* y) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
  if (!trans || ORC_MUTATE == 5) {
    /* products of every block with its column's coefficients (parallel), then
     * a serial scatter-add into the receiving rows */
    double* prod = (double*)malloc(sizeof(double) * nrows * 3 * nb);
#pragma omp parallel for schedule(static)
    for (int64_t J = 0; J < nrows; ++J)
      for (int k = 0; k < 3; ++k) {
        const double* blk = blocks + ((J * 3 + k) * (int64_t)nb) * nb;
        for (int a = 0; a < nb; ++a) {
          double s = 0.0;
          for (int b = 0; b < nb; ++b) s += blk[a * nb + b] * x[J * nb + b];
          prod[(J * 3 + k) * nb + a] = s;
        }
      }
    for (int64_t i = 0; i < nrows * nb; ++i) y[i] = x0 ? x0[i] : 0.0;
    for (int64_t J = 0; J < nrows; ++J)
      for (int k = 0; k < 3; ++k) {
        int64_t R = dest[3 * J + k];
        for (int a = 0; a < nb; ++a) y[R * nb + a] += alpha * prod[(J * 3 + k) * nb + a];
      }
    free(prod);
  } else {
#pragma omp parallel for schedule(static)
    for (int64_t J = 0; J < nrows; ++J) {
      for (int b = 0; b < nb; ++b) {
        double s = 0.0;
        for (int k = 0; k < 3; ++k) {
          int64_t R = dest[3 * J + k];
          const double* blk = blocks + ((J * 3 + k) * (int64_t)nb) * nb;
          for (int a = 0; a < nb; ++a) s += blk[a * nb + b] * x[R * nb + a];
        }
        y[J * nb + b] = (x0 ? x0[J * nb + b] : 0.0) + alpha * s;
      }
    }
  }
}
