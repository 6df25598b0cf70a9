// gates.cpp -- matrices of the circuit's gate kinds (Sect. 3).
//
// Single-qubit gates: the paper names sqrt(X), sqrt(Y), sqrt(W) without giving matrices;
// they are taken as the principal square roots sqrt(P) = exp(-i pi P / 4) = (I - i P)/sqrt 2
// with W = (X + Y)/sqrt 2.  Two-qubit gate: fSim of Eq. 1 with angles theta, phi and the
// detuning terms D+, D-, D-,off; basis index b(q0) + 2 b(q1).
#include <cmath>
#include <complex>

#include "internal.h"

namespace sycsim {

using cd = std::complex<double>;

static void put(double *out, int i, cd v)
{
    out[2 * i] = v.real();
    out[2 * i + 1] = v.imag();
}

int gate_matrix(const sim_gate &g, double *out)
{
    const cd I(0.0, 1.0);
    const double r = 1.0 / std::sqrt(2.0);
    switch (g.kind) {
    case SIM_GATE_SQRT_X:
    case SIM_GATE_SQRT_Y:
    case SIM_GATE_SQRT_W: {
        // off-diagonal entries (upper, lower) of the Pauli operator P
        cd up, lo;
        if (g.kind == SIM_GATE_SQRT_X) {
            up = 1.0;
            lo = 1.0;
        } else if (g.kind == SIM_GATE_SQRT_Y) {
            up = -I;
            lo = I;
        } else {
            up = std::exp(-I * (M_PI / 4));  // (X + Y)/sqrt 2: upper (1 - i)/sqrt 2
            lo = std::exp(I * (M_PI / 4));
        }
        put(out, 0, r);
        put(out, 1, -I * up * r);
        put(out, 2, -I * lo * r);
        put(out, 3, r);
        return 2;
    }
    case SIM_GATE_FSIM: {
        for (int i = 0; i < 32; i++) out[i] = 0.0;
        const double c = std::cos(g.theta), s = std::sin(g.theta);
        put(out, 0, 1.0);
        put(out, 1 * 4 + 1, std::exp(I * (g.dplus + g.dminus)) * c);
        put(out, 1 * 4 + 2, -I * std::exp(I * (g.dplus - g.dminus_off)) * s);
        put(out, 2 * 4 + 1, -I * std::exp(I * (g.dplus + g.dminus_off)) * s);
        put(out, 2 * 4 + 2, std::exp(I * (g.dplus - g.dminus)) * c);
        put(out, 3 * 4 + 3, std::exp(I * (2.0 * g.dplus - g.phi)));
        return 4;
    }
    case SIM_GATE_U1:
        for (int i = 0; i < 8; i++) out[i] = g.u[i];
        return 2;
    case SIM_GATE_U2:
        for (int i = 0; i < 32; i++) out[i] = g.u[i];
        return 4;
    default:
        return 0;
    }
}

}  // namespace sycsim
