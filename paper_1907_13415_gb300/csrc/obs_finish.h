// obs_finish.h -- the host-side last step of the observables, shared by
// nlc_observables (engine.cuh) and nlc_observables_static (noalloc.cu), so
// that the two entry points report the same quantities from the same grid
// totals.
#pragma once
#include <cmath>

#include "../../include/nlc.h"

namespace nlc {

// tot: the grid totals in the slot order of the observables kernels (mass,
// momentum x, y, z, sum S / s_ref, free energy, non-finite count,
// sum |u|^2, max |u|); prof[0..nx): the y, z mean of S.
//   radius (Sec. 2.2): from the nematic area A = sum S / s_ref, sqrt(A / pi)
//     on a single plane, (3 A / (4 pi))^(1/3) in 3D;
//   x_iface (Sec. 2.1): the first descending crossing of the profile through
//     s_ref / 2 (periodic in x), linearly interpolated; -1 if none.
// out->step is left to the caller.
inline void obs_from_totals(const double* tot, const double* prof, int nx, bool planar,
                            double s_ref, nlc_obs* out) {
  out->mass = tot[0];
  out->mom[0] = tot[1];
  out->mom[1] = tot[2];
  out->mom[2] = tot[3];
  out->s_area = tot[4];
  out->free_energy = tot[5];
  out->nonfinite = (int64_t)tot[6];
  out->u_l2 = std::sqrt(tot[7]);
  out->max_u = tot[8];
  out->radius = planar ? std::sqrt(tot[4] / M_PI) : std::cbrt(3.0 * tot[4] / (4.0 * M_PI));
  const double half = s_ref / 2.0;
  out->x_iface = -1.0;
  for (int x = 0; x < nx; x++) {
    const double a = prof[x], b = prof[(x + 1) % nx];
    if (a >= half && b < half) {
      out->x_iface = x + (a - half) / (a - b);
      break;
    }
  }
}

}  // namespace nlc
