// Solid-fraction laws of the latent-heat model, their slopes and the
// inversion of the enthalpy H(T) = cp T + L (1 - fs(T)):
//  * linear between T_sol and T_liq (Eq. 5 in its linear form);
//  * the Gulliver-Scheil law of Eq. 5, fs = 1 - r^(1/(kp - 1)) with
//    r = (T - T_f)/(T_liq - T_f), smeared into a straight line across
//    [T_sol - T_eps, T_sol + T_eps] so that it has a slope everywhere (Eq. 21).
// At a kink the slope is the one on the side nearer the mushy interior: the
// Scheil side at T_liq and at T_sol + T_eps, the smear side at T_sol - T_eps
// (linear law: the mushy side at both ends).
#pragma once

#include <cmath>

#include "../../include/fvs.h"

namespace fvs {

struct FsLaw {
  int scheil;    // 0 linear, 1 Eq. 21
  double Ts, Tl; // solidus, liquidus
  double Tf;     // Scheil: freezing temperature of the solvent
  double ex;     // Scheil: 1 / (kp - 1)
  double Te;     // Scheil: half-width of the smear band
};

inline FsLaw fs_law_of(const fvs_material& m) {
  FsLaw w{};
  w.scheil = m.fs_model == FVS_FS_SCHEIL ? 1 : 0;
  w.Ts = m.T_sol;
  w.Tl = m.T_liq;
  w.Tf = m.T_f;
  w.ex = w.scheil ? 1.0 / (m.kp - 1.0) : 0.0;
  w.Te = m.T_eps;
  return w;
}

// the data a law needs to be well posed with liquidus Tl
inline bool fs_law_valid(const fvs_material& m, double Tl) {
  if (m.fs_model == FVS_FS_LINEAR) return Tl > m.T_sol;
  if (m.fs_model != FVS_FS_SCHEIL) return false;
  return m.kp > 0.0 && m.kp < 1.0 && m.T_eps > 0.0 && m.T_f > Tl && Tl > m.T_sol + m.T_eps;
}

// 1 - fs on the Scheil piece
__device__ __forceinline__ double scheil_liquid(const FsLaw& w, double T) {
  return pow((T - w.Tf) / (w.Tl - w.Tf), w.ex);
}

__device__ __forceinline__ double fs_of(const FsLaw& w, double T) {
  if (!w.scheil) return fmin(fmax((w.Tl - T) / (w.Tl - w.Ts), 0.0), 1.0);
  if (T > w.Tl) return 0.0;
  const double T1 = w.Ts - w.Te, T2 = w.Ts + w.Te;
  if (T <= T1) return 1.0;
  if (T < T2) {
    const double rest = scheil_liquid(w, T2);   // 1 - fs at the top of the band
    return 1.0 - rest - (T - T2) * rest / (2.0 * w.Te);
  }
  return 1.0 - scheil_liquid(w, T);
}

__device__ __forceinline__ double fs_slope(const FsLaw& w, double T) {
  if (!w.scheil) return (T >= w.Ts && T <= w.Tl) ? -1.0 / (w.Tl - w.Ts) : 0.0;
  const double T1 = w.Ts - w.Te, T2 = w.Ts + w.Te;
  if (T > w.Tl || T < T1) return 0.0;
  if (T < T2) return -scheil_liquid(w, T2) / (2.0 * w.Te);
  const double r = (T - w.Tf) / (w.Tl - w.Tf);
  return -w.ex * pow(r, w.ex - 1.0) / (w.Tl - w.Tf);
}

// the temperature whose enthalpy cp T + L (1 - fs(T)) is H (strictly
// increasing in T): closed form on the solid, liquid, linear and smear
// pieces; on the Scheil piece g(T) = cp T + L r^ex - H is increasing and
// convex, so Newton's method started at T_liq descends onto the root without
// overshooting (bounded at 100 steps)
__device__ __forceinline__ double T_of_H(const FsLaw& w, double cp, double L, double H) {
  if (!w.scheil) {
    const double Hs = cp * w.Ts, Hl = cp * w.Tl + L;
    if (H <= Hs) return H / cp;
    if (H >= Hl) return (H - L) / cp;
    return w.Ts + (H - Hs) / (Hl - Hs) * (w.Tl - w.Ts);
  }
  const double T1 = w.Ts - w.Te, T2 = w.Ts + w.Te;
  const double H1 = cp * T1, H2 = cp * T2 + L * scheil_liquid(w, T2), H3 = cp * w.Tl + L;
  if (H <= H1) return H / cp;
  if (H >= H3) return (H - L) / cp;
  if (H < H2) return T1 + (H - H1) / (H2 - H1) * (T2 - T1);
  const double span = w.Tl - w.Tf;
  double T = w.Tl;
  for (int it = 0; it < 100; ++it) {
    const double r = (T - w.Tf) / span;
    const double q = pow(r, w.ex);
    const double g = cp * T + L * q - H;
    const double dg = cp + L * w.ex * q / (r * span);
    const double step = g / dg;
    T -= step;
    if (fabs(step) <= 1e-12) break;
  }
  return fmin(fmax(T, T2), w.Tl);
}

}  // namespace fvs
