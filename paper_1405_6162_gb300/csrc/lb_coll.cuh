// lb_coll.cuh -- the collision's parameter structs in the arithmetic type,
// formed on the host in double and rounded once.
#pragma once

#include "d3q19.cuh"
#include "lb.h"

namespace lbk {

// Parameters of the step in the arithmetic type T (constants formed in
// double, rounded once).
template <typename T>
inline Coll<T> make_coll(const lb_params &p)
{
    const double om = 1.0 / p.tau, og = 1.0 / p.tau_g;
    Coll<T> c;
    c.omega = T(om);
    c.omega_g = T(og);
    c.rho0 = T(p.rho0);
    c.gamma = T(p.gamma);
    c.A = T(p.A);
    c.B = T(p.B);
    c.kappa = T(p.kappa);
    c.hA = T(0.5 * p.A);
    c.qB = T(0.75 * p.B);
    c.cf = T(1.0 - om);
    c.f0 = T(om / 3.0);  c.f1 = T(om / 18.0);  c.f2 = T(om / 36.0);
    c.f1h = T(om / 4.0); c.f2h = T(om / 8.0);
    c.f1t = T(om / 6.0); c.f2t = T(om / 12.0);
    c.cg = T(1.0 - og);
    c.g0 = T(og / 3.0);  c.g1 = T(og / 18.0);  c.g2 = T(og / 36.0);
    c.g1h = T(og / 4.0); c.g2h = T(og / 8.0);
    c.g1t = T(og / 6.0); c.g2t = T(og / 12.0);
    return c;
}

// MRT rates and body force in the arithmetic type T (mrt = 0: BGK with a
// force, all three rates 1/tau -- Guo's BGK scheme)
template <typename T>
inline Mrt<T> make_mrt(const lb_params &p, bool mrt, double tau_bulk, double tau_ghost, const double *force)
{
    const double ws = 1.0 / p.tau;
    const double wb = mrt ? 1.0 / tau_bulk : ws, wg = mrt ? 1.0 / tau_ghost : ws;
    Mrt<T> m;
    m.cs = T(1.0 - ws);
    m.cb = T(1.0 - wb);
    m.hs = T(1.0 - 0.5 * ws);
    m.hb = T(1.0 - 0.5 * wb);
    m.og = T(wg);
    m.cgh = T(1.0 - wg);
    m.kf = T(1.0 - 0.5 * wg);
    m.Fx = T(force[0]);
    m.Fy = T(force[1]);
    m.Fz = T(force[2]);
    m.hFx = T(0.5 * force[0]);
    m.hFy = T(0.5 * force[1]);
    m.hFz = T(0.5 * force[2]);
    return m;
}

}  // namespace lbk
