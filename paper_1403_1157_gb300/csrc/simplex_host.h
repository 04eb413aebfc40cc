// Host helpers shared by the simplicial operators (tri.cu, tet.cu).
#pragma once

namespace cdg2 {

// Jacobi P_n^{(a,0)} and its derivative at x (three-term recurrence, DLMF
// 18.9.1 with beta = 0, and its derivative).
inline void jacobi_d(int n, double a, double x, double& P, double& dP) {
    double p0 = 1.0, d0 = 0.0;
    if (n == 0) {
        P = p0;
        dP = d0;
        return;
    }
    double p1 = (a + 1.0) + (a + 2.0) * (x - 1.0) / 2.0, d1 = (a + 2.0) / 2.0;
    for (int m = 2; m <= n; ++m) {
        const double c = 2.0 * m + a;
        const double a1 = 2.0 * m * (m + a) * (c - 2.0);
        const double a2 = (c - 1.0) * c * (c - 2.0);
        const double a3 = (c - 1.0) * a * a;
        const double a4 = 2.0 * (m + a - 1.0) * (m - 1.0) * c;
        const double p2 = ((a2 * x + a3) * p1 - a4 * p0) / a1;
        const double d2 = ((a2 * x + a3) * d1 + a2 * p1 - a4 * d0) / a1;
        p0 = p1;
        d0 = d1;
        p1 = p2;
        d1 = d2;
    }
    P = p1;
    dP = d1;
}

}  // namespace cdg2
