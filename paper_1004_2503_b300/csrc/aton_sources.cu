// aton_sources.cu -- host source model of the post-processing (section 2.3): star particles
// of the next snapshot turned into nearest-grid-point emission rates spread over the snapshot
// interval, with the escape fraction and the resolution boost factor (Eqs. 16-17). Host code:
// a per-star recipe evaluated once per snapshot interval; the result feeds aton_add_sources.
#include <cmath>
#include <cstdint>

#include "aton_internal.h"

namespace {

constexpr double kMH = 1.6735575e-24;   // hydrogen atom mass [g] (one baryon)

int wrap(double x, double dx, int n) {
  long long i = (long long)std::floor(x / dx);
  i %= n;
  if (i < 0) i += n;
  return (int)i;
}

}  // namespace

int aton_star_sources(const aton_star* stars, int64_t n, const aton_source_model* m, int nx,
                      int ny, int nz, double dx, int64_t* cell, double* rate) {
  if (n < 0) {
    aton::set_last_message("n < 0");
    return ATON_ERR_BADARG;
  }
  if (n > 0 && (!stars || !cell || !rate)) {
    aton::set_last_message("NULL array");
    return ATON_ERR_BADARG;
  }
  if (!m || nx < 1 || ny < 1 || nz < 1 || !(dx > 0.0) || !std::isfinite(dx)) {
    aton::set_last_message("bad model or grid");
    return ATON_ERR_BADARG;
  }
  const double D = m->interval;
  if (!(D > 0.0) || !std::isfinite(D) || !(m->f_esc >= 0.0) || !std::isfinite(m->f_esc) ||
      !(m->t_universe > 0.0) || !std::isfinite(m->boost_a) || !std::isfinite(m->boost_k)) {
    aton::set_last_message("bad source model (interval, f_esc, t_universe, boost)");
    return ATON_ERR_BADARG;
  }
  const double B =
      m->boost_a > 0.0 ? std::fmax(1.0, m->boost_a * std::exp(m->boost_k / m->t_universe)) : 1.0;
  const double k = m->f_esc * B;
  for (int64_t s = 0; s < n; ++s) {
    const aton_star& st = stars[s];
    if (!(st.mass >= 0.0) || !std::isfinite(st.mass) || !(st.age >= 0.0) ||
        !std::isfinite(st.age) || !(st.lifetime > 0.0) || !std::isfinite(st.lifetime) ||
        !(st.photons_per_baryon >= 0.0) || !std::isfinite(st.photons_per_baryon) ||
        !std::isfinite(st.x) || !std::isfinite(st.y) || !std::isfinite(st.z)) {
      aton::set_last_message("invalid star record");
      return ATON_ERR_BADARG;
    }
    const double L = st.lifetime, a = st.age, ap = a - D;
    double emit;   // emitting time inside the interval
    if (ap >= L) emit = 0.0;
    else if (ap < 0.0) emit = std::fmin(a, L);
    else emit = std::fmin(D, L - ap);
    const double ndot = st.photons_per_baryon * st.mass / kMH / L;
    if (!(emit > 0.0)) {
      cell[s] = -1;
      rate[s] = 0.0;
      continue;
    }
    const int i = wrap(st.x, dx, nx), j = wrap(st.y, dx, ny), kk = wrap(st.z, dx, nz);
    cell[s] = (int64_t)i + (int64_t)nx * ((int64_t)j + (int64_t)ny * kk);
    rate[s] = emit / D * ndot * k;
  }
  return ATON_OK;
}
