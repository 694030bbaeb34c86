// Host-side set-up of a material's device form (MatDev, common.cuh): the
// spline's cubic Hermite segment coefficients and rest-state expansion
// constants, and the copy of a checked host material.
#pragma once

#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "setup.hpp"

namespace hqn {

// Value and derivative at t of the C1 cubic Hermite interpolant of knots x,
// values v and slopes m, continued quadratically outside [x0, x7].
inline void hermite_at(const double *x, const double *v, const double *m, double t, double &val, double &der) {
    const double tc = std::min(std::max(t, x[0]), x[7]);
    int i = 0;
    for (int k = 1; k < 7; ++k)
        if (tc >= x[k]) i = k;
    const double h = x[i + 1] - x[i], u = (tc - x[i]) / h;
    const double m0 = m[i] * h, m1 = m[i + 1] * h;
    const double c2 = 3.0 * (v[i + 1] - v[i]) - 2.0 * m0 - m1, c3 = 2.0 * (v[i] - v[i + 1]) + m0 + m1;
    const double pv = v[i] + u * (m0 + u * (c2 + u * c3));
    const double pd = (m0 + u * (2.0 * c2 + 3.0 * u * c3)) / h;
    const double p2 = (2.0 * c2 + 6.0 * u * c3) / (h * h);
    const double dt = t - tc;
    val = pv + dt * (pd + 0.5 * p2 * dt);
    der = pd + p2 * dt;
}

// Fills the spline part of d from knots sx, values sv and slopes ss of the
// functions a, b, c (knots strictly increasing).
template <typename R>
void fill_spline(MatDev<R> &d, const double sx[3][8], const double sv[3][8], const double ss[3][8]) {
    double F0[3], F1[3];
    for (int f = 0; f < 3; ++f) {
        hermite_at(sx[f], sv[f], ss[f], 1.0, F0[f], F1[f]);
        for (int i = 0; i < 8; ++i) d.kx[f][i] = (R)(sx[f][i] - 1.0);
        for (int i = 0; i < 7; ++i) {
            const double h = sx[f][i + 1] - sx[f][i];
            const double v0 = sv[f][i], v1 = sv[f][i + 1];
            const double m0 = ss[f][i] * h, m1 = ss[f][i + 1] * h;
            d.inv_h[f][i] = (R)(1.0 / h);
            d.p[f][i][0] = (R)v0;
            d.p[f][i][1] = (R)m0;
            d.p[f][i][2] = (R)(3.0 * (v1 - v0) - 2.0 * m0 - m1);
            d.p[f][i][3] = (R)(2.0 * (v0 - v1) + m0 + m1);
            // the segment's point nearest the rest state t = 1
            const double ref = std::min(std::max(1.0, sx[f][i]), sx[f][i + 1]);
            double fv, fd;
            hermite_at(sx[f], sv[f], ss[f], ref, fv, fd);
            d.ur[f][i] = (R)((ref - sx[f][i]) / h);
            d.dD[f][i] = (R)(fd - F1[f]);
            d.dE[f][i] = (R)(fv - F0[f] - F1[f] * (ref - 1.0));
        }
    }
    d.K0 = (R)(F1[0] + 2.0 * F1[1] + F1[2]);
    d.B1C1 = (R)(F1[1] + F1[2]);
    d.C1 = (R)F1[2];
    d.psi_rest = (R)(3.0 * F0[0] + 3.0 * F0[1] + F0[2]);
}

// The kernel form of a checked host material (material_from_api).
template <typename R>
void matdev_from_host(const MaterialHost &m, MatDev<R> &M) {
    M = MatDev<R>{};
    M.kind = m.kind;
    M.mu = (R)m.mu;
    M.lam = (R)m.lam;
    M.J0 = (R)m.J0;
    M.c0 = (R)m.c0;
    M.c1 = (R)m.c1;
    M.c2 = (R)m.c2;
    if (m.kind == HQN_SPLINE_VL) fill_spline(M, m.sx, m.sv, m.ss);
    M.kappa = (R)m.kappa;
    for (int a = 0; a < 3; ++a) M.fd[a] = (R)m.fiber[a];
}

}  // namespace hqn
