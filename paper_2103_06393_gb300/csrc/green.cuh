// Coupling-matrix entries from the free-space Green's function (Sec. III.A; Eq. n6, Eq. nNt,
// Eq. nKt), FP64.
//
// Point-matched at the segment centre (green_entry, the N operator):
//   Z[(k,v), e] = h^3 len_e [ (I + grad grad / k0^2) g(r_v - c_e) t_e ]_k with
// g = exp(-i k0 R)/(4 pi R) and, for x = k0 R and Rhat = (r_v - c_e)/R,
//   (I + grad grad/k0^2) g = g [ (1 - i/x - 1/x^2) I + (-1 + 3i/x + 3/x^2) Rhat Rhat^T ].
// With an nq-point Gauss-Legendre rule along the segment (segment_entry), the N or the K operator:
//   Z[(k,v), e] = h^3 len_e sum_q (w_q / 2) [ Kern(r_v - p_q) t_e ]_k,  p_q = c_e + xi_q len_e t_e / 2,
//   K: Kern t = grad g x t = g' (Rhat x t),  g' = -g (i k0 + 1/R).
#pragma once

#include <cmath>

#include "zbc_internal.cuh"

namespace zbc {

constexpr int kMaxQuad = 16;  // Gauss-Legendre points per segment, at most

struct GreenGeom {
  int n1, n2, n3;
  double h, mask_r, mask_b, k0;
  const double* centre;
  const double* tangent;
  const double* length;
  int m;
  int op;                   // 0: N operator (Eq. nNt), 1: K operator (Eq. nKt)
  int nq;                   // quadrature points along the segment
  double qx[kMaxQuad];      // nodes on [-1, 1]
  double qw[kMaxQuad];      // weights (sum 2)
};

// voxel centre (same rounding as ((i - (n-1)/2) * h)) and the mask decision
__device__ __forceinline__ bool voxel_centre(const GreenGeom& G, int64_t v, double& x, double& y, double& z) {
  const int i1 = (int)(v % G.n1);
  const int i2 = (int)((v / G.n1) % G.n2);
  const int i3 = (int)(v / ((int64_t)G.n1 * G.n2));
  x = __dmul_rn((double)i1 - (G.n1 - 1) / 2.0, G.h);
  y = __dmul_rn((double)i2 - (G.n2 - 1) / 2.0, G.h);
  z = __dmul_rn((double)i3 - (G.n3 - 1) / 2.0, G.h);
  if (G.mask_b > 0.0 && (fabs(x) > G.mask_b || fabs(y) > G.mask_b)) return false;
  if (G.mask_r > 0.0) return !(sqrt(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y))) > G.mask_r);
  return true;
}

// the three components of Z[(., v), e]; zero for masked voxels or e outside [0, m)
__device__ __forceinline__ void green_entry(const GreenGeom& G, int64_t v, int e, double2 (&out)[3]) {
  double x, y, z;
  const bool keep = voxel_centre(G, v, x, y, z) && e >= 0 && e < G.m;
#pragma unroll
  for (int k = 0; k < 3; ++k) out[k] = make_double2(0.0, 0.0);
  if (!keep) return;
  const double Rx = x - G.centre[3 * e + 0], Ry = y - G.centre[3 * e + 1], Rz = z - G.centre[3 * e + 2];
  const double R = sqrt(Rx * Rx + Ry * Ry + Rz * Rz);
  const double iR = 1.0 / R;
  const double hx = Rx * iR, hy = Ry * iR, hz = Rz * iR;
  const double tx = G.tangent[3 * e + 0], ty = G.tangent[3 * e + 1], tz = G.tangent[3 * e + 2];
  const double kr = G.k0 * R, ikr = 1.0 / kr, ikr2 = ikr * ikr;
  double s, c;
  sincos(kr, &s, &c);
  const double scale = G.h * G.h * G.h * G.length[e] / (4.0 * M_PI * R);
  const double gr = scale * c, gi = -scale * s;  // scale * exp(-i kR)
  const double ar = 1.0 - ikr2, ai = -ikr;        // 1 - i/x - 1/x^2
  const double br = -1.0 + 3.0 * ikr2, bi = 3.0 * ikr;  // -1 + 3i/x + 3/x^2
  const double ht = hx * tx + hy * ty + hz * tz;
  const double tk[3] = {tx, ty, tz}, hk[3] = {hx, hy, hz};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double ur = ar * tk[k] + br * hk[k] * ht;
    const double ui = ai * tk[k] + bi * hk[k] * ht;
    out[k] = make_double2(gr * ur - gi * ui, gr * ui + gi * ur);
  }
}

// sum over the segment's quadrature points of (w_q / 2) Kern(r - p_q) t_e at the point r
// (without the h^3 len_e factor): accr, acci hold the three components
__device__ __forceinline__ void field_at(const GreenGeom& G, double x, double y, double z, int e, double (&accr)[3],
                                         double (&acci)[3]) {
  const double tx = G.tangent[3 * e + 0], ty = G.tangent[3 * e + 1], tz = G.tangent[3 * e + 2];
  const double len = G.length[e];
#pragma unroll
  for (int k = 0; k < 3; ++k) accr[k] = acci[k] = 0.0;
  for (int iq = 0; iq < G.nq; ++iq) {
    const double off = 0.5 * G.qx[iq] * len;
    const double Rx = x - (G.centre[3 * e + 0] + off * tx), Ry = y - (G.centre[3 * e + 1] + off * ty),
                 Rz = z - (G.centre[3 * e + 2] + off * tz);
    const double R = sqrt(Rx * Rx + Ry * Ry + Rz * Rz);
    const double iR = 1.0 / R;
    const double hx = Rx * iR, hy = Ry * iR, hz = Rz * iR;
    double s, c;
    sincos(G.k0 * R, &s, &c);
    const double wq = 0.5 * G.qw[iq] / (4.0 * M_PI * R);
    const double gr = wq * c, gi = -wq * s;  // (w_q / 2) g
    double ur[3], ui[3];
    if (G.op == 0) {
      const double kr = G.k0 * R, ikr = 1.0 / kr, ikr2 = ikr * ikr;
      const double ar = 1.0 - ikr2, ai = -ikr, br = -1.0 + 3.0 * ikr2, bi = 3.0 * ikr;
      const double ht = hx * tx + hy * ty + hz * tz;
      const double tk[3] = {tx, ty, tz}, hk[3] = {hx, hy, hz};
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        ur[k] = ar * tk[k] + br * hk[k] * ht;
        ui[k] = ai * tk[k] + bi * hk[k] * ht;
      }
    } else {
      // g' / g = -(i k0 + 1/R) = -1/R - i k0; Rhat x t
      const double cx = hy * tz - hz * ty, cy = hz * tx - hx * tz, cz = hx * ty - hy * tx;
      const double pr = -iR, pi = -G.k0;
      const double ck[3] = {cx, cy, cz};
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        ur[k] = pr * ck[k];
        ui[k] = pi * ck[k];
      }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      accr[k] += gr * ur[k] - gi * ui[k];
      acci[k] += gr * ui[k] + gi * ur[k];
    }
  }
}

// the three components at the voxel centre, times h^3 len_e; zero for masked voxels or e
// outside [0, m)
__device__ __forceinline__ void segment_entry(const GreenGeom& G, int64_t v, int e, double2 (&out)[3]) {
  double x, y, z;
  const bool keep = voxel_centre(G, v, x, y, z) && e >= 0 && e < G.m;
#pragma unroll
  for (int k = 0; k < 3; ++k) out[k] = make_double2(0.0, 0.0);
  if (!keep) return;
  double fr[3], fi[3];
  field_at(G, x, y, z, e, fr, fi);
  const double sc = G.h * G.h * G.h * G.length[e];
#pragma unroll
  for (int k = 0; k < 3; ++k) out[k] = make_double2(sc * fr[k], sc * fi[k]);
}

// piecewise-linear basis (q = 12): phi_0 = 1, phi_1..3 = (x - x_c)/h, (y - y_c)/h, (z - z_c)/h,
// integrated over the voxel with the 2 x 2 x 2 Gauss-Legendre rule (points at offsets
// +-h / (2 sqrt 3) per axis, weights 1/8), times h^3 len_e; out[3 l + k] for basis l, component k
__device__ __forceinline__ void pwl_entry(const GreenGeom& G, int64_t v, int e, double2 (&out)[12]) {
  double x, y, z;
  const bool keep = voxel_centre(G, v, x, y, z) && e >= 0 && e < G.m;
#pragma unroll
  for (int b = 0; b < 12; ++b) out[b] = make_double2(0.0, 0.0);
  if (!keep) return;
  const double a = 0.5 / sqrt(3.0);  // offset / h of the 2-point rule on [-1/2, 1/2]
  for (int pt = 0; pt < 8; ++pt) {
    const double dx = (pt & 1) ? a : -a, dy = (pt & 2) ? a : -a, dz = (pt & 4) ? a : -a;
    double fr[3], fi[3];
    field_at(G, x + G.h * dx, y + G.h * dy, z + G.h * dz, e, fr, fi);
    const double phi[4] = {1.0, dx, dy, dz};
#pragma unroll
    for (int l = 0; l < 4; ++l)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        out[3 * l + k].x += 0.125 * phi[l] * fr[k];
        out[3 * l + k].y += 0.125 * phi[l] * fi[k];
      }
  }
  const double sc = G.h * G.h * G.h * G.length[e];
#pragma unroll
  for (int b = 0; b < 12; ++b) out[b] = make_double2(sc * out[b].x, sc * out[b].y);
}

inline double wavenumber(double freq_hz) { return 2.0 * M_PI * freq_hz / 299792458.0; }

// nq-point Gauss-Legendre rule on [-1, 1]: the roots of P_nq by Newton's method from the
// Chebyshev-like first guesses cos(pi (i - 1/4) / (nq + 1/2)), weights 2 / ((1 - x^2) P'_nq(x)^2)
inline void gauss_legendre(int nq, double* x, double* w) {
  for (int i = 0; i < nq; ++i) {
    double xi = std::cos(M_PI * (i + 0.75) / (nq + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = xi;  // P_0, P_1
      for (int k = 2; k <= nq; ++k) {
        const double pk = ((2.0 * k - 1.0) * xi * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = pk;
      }
      dp = nq * (xi * p1 - p0) / (xi * xi - 1.0);  // P'_nq from P_nq and P_nq-1
      const double dx = p1 / dp;
      xi -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    x[i] = xi;
    w[i] = 2.0 / ((1.0 - xi * xi) * dp * dp);
  }
}

}  // namespace zbc
