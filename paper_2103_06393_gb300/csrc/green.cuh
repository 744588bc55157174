// Coupling-matrix entries from the dyadic Green's function (Sec. III.A; Eq. n6, Eq. nNt), FP64.
//
// Z[(k,v), e] = h^3 len_e [ (I + grad grad / k0^2) g(r_v - c_e) t_e ]_k with
// g = exp(-i k0 R)/(4 pi R) and, for x = k0 R and Rhat = (r_v - c_e)/R,
//   (I + grad grad/k0^2) g = g [ (1 - i/x - 1/x^2) I + (-1 + 3i/x + 3/x^2) Rhat Rhat^T ].
#pragma once

#include <cmath>

#include "zbc_internal.cuh"

namespace zbc {

struct GreenGeom {
  int n1, n2, n3;
  double h, mask_r, k0;
  const double* centre;
  const double* tangent;
  const double* length;
  int m;
};

// voxel centre (same rounding as ((i - (n-1)/2) * h)) and the mask decision
__device__ __forceinline__ bool voxel_centre(const GreenGeom& G, int64_t v, double& x, double& y, double& z) {
  const int i1 = (int)(v % G.n1);
  const int i2 = (int)((v / G.n1) % G.n2);
  const int i3 = (int)(v / ((int64_t)G.n1 * G.n2));
  x = __dmul_rn((double)i1 - (G.n1 - 1) / 2.0, G.h);
  y = __dmul_rn((double)i2 - (G.n2 - 1) / 2.0, G.h);
  z = __dmul_rn((double)i3 - (G.n3 - 1) / 2.0, G.h);
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

inline double wavenumber(double freq_hz) { return 2.0 * M_PI * freq_hz / 299792458.0; }

}  // namespace zbc
