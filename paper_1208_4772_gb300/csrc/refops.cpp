// Host FP64 construction of the reference operators (see refops.h).
#include "refops.h"

#include <algorithm>
#include <cmath>

namespace dgc {

namespace detail {

// Orthonormal Jacobi polynomial of degree n for the weight (1-x)^a (1+x)^b,
// by the three-term recurrence of the orthonormal family
//   x p_n = A_{n+1} p_{n+1} + B_n p_n + A_n p_{n-1}.
double jac(double x, double a, double b, int n) {
    const double ab = a + b;
    const double h0 = std::pow(2.0, ab + 1.0) * std::tgamma(a + 1.0) * std::tgamma(b + 1.0) /
                      std::tgamma(ab + 2.0);
    double p_prev = 1.0 / std::sqrt(h0);
    if (n == 0) return p_prev;
    const double A1 = 2.0 / (ab + 2.0) * std::sqrt((a + 1.0) * (b + 1.0) / (ab + 3.0));
    const double B0 = (ab == 0.0) ? 0.0 : (b * b - a * a) / (ab * (ab + 2.0));
    double p = (x - B0) * p_prev / A1;
    double A_old = A1;
    for (int i = 1; i < n; ++i) {
        const double c = 2.0 * i + ab;
        const double A_new = 2.0 / (c + 2.0) *
            std::sqrt((i + 1.0) * (i + 1.0 + ab) * (i + 1.0 + a) * (i + 1.0 + b) / ((c + 1.0) * (c + 3.0)));
        const double Bi = (b * b - a * a) / (c * (c + 2.0));
        const double p_next = ((x - Bi) * p - A_old * p_prev) / A_new;
        p_prev = p;
        p = p_next;
        A_old = A_new;
    }
    return p;
}

// d/dx of the orthonormal polynomial: sqrt(n (n+a+b+1)) p_{n-1}^{(a+1,b+1)}.
double djac(double x, double a, double b, int n) {
    if (n == 0) return 0.0;
    return std::sqrt(n * (n + a + b + 1.0)) * jac(x, a + 1.0, b + 1.0, n - 1);
}

// Gauss rule for the weight (1-x)^a (1+x)^b: Newton with deflation for the
// roots, Christoffel numbers 1 / sum_m p_m(x)^2 for the weights.
void gauss_jacobi(int n, double a, double b, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int k = 0; k < n; ++k) {
        double xk = -std::cos((2.0 * k + 1.0) * M_PI / (2.0 * n));
        if (k > 0) xk = 0.5 * (xk + x[k - 1]);
        for (int it = 0; it < 200; ++it) {
            const double p = jac(xk, a, b, n), dp = djac(xk, a, b, n);
            double s = 0.0;
            for (int j = 0; j < k; ++j) s += 1.0 / (xk - x[j]);
            const double dx = p / (dp - p * s);
            xk -= dx;
            if (std::fabs(dx) < 1e-16) break;
        }
        x[k] = xk;
    }
    std::sort(x.begin(), x.end());
    for (int k = 0; k < n; ++k) {
        double s = 0.0;
        for (int m = 0; m < n; ++m) {
            const double p = jac(x[k], a, b, m);
            s += p * p;
        }
        w[k] = 1.0 / s;
    }
}

std::vector<double> gll(int N) {
    std::vector<double> x(N + 1);
    x[0] = -1.0;
    x[N] = 1.0;
    if (N >= 2) {
        std::vector<double> xi, wi;
        gauss_jacobi(N - 1, 1.0, 1.0, xi, wi);
        for (int i = 0; i < N - 1; ++i) x[i + 1] = xi[i];
    }
    return x;
}

// Warp & blend nodes (blending parameter 0) in the canonical order.
void nodes_2d(int N, std::vector<double>& r, std::vector<double>& s) {
    const int Np = n_modes(N);
    r.assign(Np, 0.0);
    s.assign(Np, 0.0);
    const double q3 = std::sqrt(3.0);
    const double A[2] = {-1.0, -1.0 / q3}, B[2] = {1.0, -1.0 / q3}, C[2] = {0.0, 2.0 / q3};
    const std::vector<double> xg = gll(N);
    std::vector<double> xe(N + 1);
    for (int i = 0; i <= N; ++i) xe[i] = -1.0 + 2.0 * i / N;
    auto warp = [&](double t) {
        if (std::fabs(t) >= 1.0 - 1e-10) return 0.0;
        double w = 0.0;
        for (int i = 0; i <= N; ++i) {
            double l = 1.0;
            for (int m = 0; m <= N; ++m)
                if (m != i) l *= (t - xe[m]) / (xe[i] - xe[m]);
            w += (xg[i] - xe[i]) * l;
        }
        return w / (1.0 - t * t);
    };
    int n = 0;
    for (int j = 0; j <= N; ++j) {
        for (int i = 0; i <= N - j; ++i, ++n) {
            const double lB = double(i) / N, lC = double(j) / N, lA = 1.0 - lB - lC;
            double lam[3] = {lA, lB, lC};
            const double* P[3] = {A, B, C};
            double X = lA * A[0] + lB * B[0] + lC * C[0];
            double Y = lA * A[1] + lB * B[1] + lC * C[1];
            for (int e = 0; e < 3; ++e) {
                const int p = e, qn = (e + 1) % 3;
                const double dx = P[qn][0] - P[p][0], dy = P[qn][1] - P[p][1];
                const double len = std::sqrt(dx * dx + dy * dy);
                const double f = 4.0 * lam[p] * lam[qn] * warp(lam[qn] - lam[p]);
                X += f * dx / len;
                Y += f * dy / len;
            }
            // barycentrics of (X, Y) on the equilateral triangle
            const double det = (B[0] - A[0]) * (C[1] - A[1]) - (C[0] - A[0]) * (B[1] - A[1]);
            const double mB = ((X - A[0]) * (C[1] - A[1]) - (C[0] - A[0]) * (Y - A[1])) / det;
            const double mC = ((B[0] - A[0]) * (Y - A[1]) - (X - A[0]) * (B[1] - A[1])) / det;
            const double mA = 1.0 - mB - mC;
            r[n] = -mA + mB - mC;
            s[n] = -mA - mB + mC;
        }
    }
}

// Modes in hierarchical order: total degree d, then i; (i, j = d - i).
void mode_ij(int N, std::vector<int>& I, std::vector<int>& J) {
    I.clear();
    J.clear();
    for (int d = 0; d <= N; ++d)
        for (int i = 0; i <= d; ++i) {
            I.push_back(i);
            J.push_back(d - i);
        }
}

// psi_ij and its (r, s) gradient at one point; collapsed a = 2(1+r)/(1-s)-1.
void psi(int i, int j, double r, double s, double* val, double* dr, double* ds) {
    const double b = s;
    const double a = (std::fabs(1.0 - s) > 1e-14) ? 2.0 * (1.0 + r) / (1.0 - s) - 1.0 : -1.0;
    const double fa = jac(a, 0.0, 0.0, i), dfa = djac(a, 0.0, 0.0, i);
    const double gb = jac(b, 2.0 * i + 1.0, 0.0, j), dgb = djac(b, 2.0 * i + 1.0, 0.0, j);
    const double om = 1.0 - b;
    const double omi = std::pow(om, i);
    const double r2 = std::sqrt(2.0);
    if (val) *val = r2 * fa * gb * omi;
    if (dr || ds) {
        // (d psi / da) / (1 - b) without dividing by zero for i = 0
        const double da_over = (i > 0) ? dfa * gb * std::pow(om, i - 1) : 0.0;
        double db = fa * dgb * omi;
        if (i > 0) db -= i * fa * gb * std::pow(om, i - 1);
        if (dr) *dr = r2 * 2.0 * da_over;
        if (ds) *ds = r2 * ((1.0 + a) * da_over + db);
    }
}

void matmul(const std::vector<double>& A, const std::vector<double>& B, std::vector<double>& C,
            int n, int k, int m) {
    C.assign((size_t)n * m, 0.0);
    for (int i = 0; i < n; ++i)
        for (int l = 0; l < k; ++l) {
            const double a = A[(size_t)i * k + l];
            for (int j = 0; j < m; ++j) C[(size_t)i * m + j] += a * B[(size_t)l * m + j];
        }
}

}  // namespace detail

using namespace detail;

int default_q(int N) { return (3 * N + 2) / 2; }
int n_modes(int N) { return (N + 1) * (N + 2) / 2; }

bool invert(std::vector<double>& A, int n) {
    std::vector<double> I((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) I[(size_t)i * n + i] = 1.0;
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int i = c + 1; i < n; ++i)
            if (std::fabs(A[(size_t)i * n + c]) > std::fabs(A[(size_t)piv * n + c])) piv = i;
        if (A[(size_t)piv * n + c] == 0.0) return false;
        if (piv != c)
            for (int j = 0; j < n; ++j) {
                std::swap(A[(size_t)c * n + j], A[(size_t)piv * n + j]);
                std::swap(I[(size_t)c * n + j], I[(size_t)piv * n + j]);
            }
        const double d = 1.0 / A[(size_t)c * n + c];
        for (int j = 0; j < n; ++j) {
            A[(size_t)c * n + j] *= d;
            I[(size_t)c * n + j] *= d;
        }
        for (int i = 0; i < n; ++i) {
            if (i == c) continue;
            const double f = A[(size_t)i * n + c];
            if (f == 0.0) continue;
            for (int j = 0; j < n; ++j) {
                A[(size_t)i * n + j] -= f * A[(size_t)c * n + j];
                I[(size_t)i * n + j] -= f * I[(size_t)c * n + j];
            }
        }
    }
    A.swap(I);
    return true;
}

bool spd_inverse(const double* A, double* Ainv, int n) {
    // A = L L^T, then A^-1 = L^-T L^-1
    std::vector<double> L((size_t)n * n, 0.0);
    for (int j = 0; j < n; ++j) {
        double d = A[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) d -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
        if (!(d > 0.0)) return false;
        d = std::sqrt(d);
        L[(size_t)j * n + j] = d;
        for (int i = j + 1; i < n; ++i) {
            double v = A[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) v -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
            L[(size_t)i * n + j] = v / d;
        }
    }
    // Linv lower triangular
    std::vector<double> Li((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) {
        Li[(size_t)i * n + i] = 1.0 / L[(size_t)i * n + i];
        for (int j = 0; j < i; ++j) {
            double v = 0.0;
            for (int k = j; k < i; ++k) v -= L[(size_t)i * n + k] * Li[(size_t)k * n + j];
            Li[(size_t)i * n + j] = v / L[(size_t)i * n + i];
        }
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double v = 0.0;
            for (int k = std::max(i, j); k < n; ++k) v += Li[(size_t)k * n + i] * Li[(size_t)k * n + j];
            Ainv[(size_t)i * n + j] = v;
        }
    return true;
}

bool build_refops(int N, int q, RefOps& o, std::string& err) {
    if (N < 1 || N > 8) {
        err = "degree N out of range";
        return false;
    }
    if (q <= 0) q = default_q(N);
    o.N = N;
    o.Np = n_modes(N);
    o.q = q;
    o.Nq = q * q;
    o.Ng = q;
    o.Nf = 3 * q;
    const int Np = o.Np, Nq = o.Nq, Ng = o.Ng, Nf = o.Nf;

    nodes_2d(N, o.r, o.s);
    std::vector<int> I, J;
    mode_ij(N, I, J);
    o.degree.resize(Np);
    for (int m = 0; m < Np; ++m) o.degree[m] = I[m] + J[m];

    o.V.assign((size_t)Np * Np, 0.0);
    for (int i = 0; i < Np; ++i)
        for (int m = 0; m < Np; ++m) psi(I[m], J[m], o.r[i], o.s[i], &o.V[(size_t)i * Np + m], nullptr, nullptr);
    o.Vinv = o.V;
    if (!invert(o.Vinv, Np)) {
        err = "singular Vandermonde matrix";
        return false;
    }

    // volume rule: Gauss-Legendre in a times Gauss-Jacobi(1,0) in b
    std::vector<double> a, wa, b, wb;
    gauss_jacobi(q, 0.0, 0.0, a, wa);
    gauss_jacobi(q, 1.0, 0.0, b, wb);
    o.rq.resize(Nq);
    o.sq.resize(Nq);
    o.wq.resize(Nq);
    for (int j = 0; j < q; ++j)
        for (int i = 0; i < q; ++i) {
            const int n = j * q + i;
            o.rq[n] = 0.5 * (1.0 + a[i]) * (1.0 - b[j]) - 1.0;
            o.sq[n] = b[j];
            o.wq[n] = 0.5 * wa[i] * wb[j];
        }
    o.tg = a;
    o.wg = wa;

    auto build = [&](const std::vector<double>& pr, const std::vector<double>& ps, std::vector<double>& Iout,
                     std::vector<double>& Drout, std::vector<double>& Dsout) {
        const int n = (int)pr.size();
        std::vector<double> Vp((size_t)n * Np), Vr((size_t)n * Np), Vs((size_t)n * Np);
        for (int i = 0; i < n; ++i)
            for (int m = 0; m < Np; ++m)
                psi(I[m], J[m], pr[i], ps[i], &Vp[(size_t)i * Np + m], &Vr[(size_t)i * Np + m],
                    &Vs[(size_t)i * Np + m]);
        matmul(Vp, o.Vinv, Iout, n, Np, Np);
        matmul(Vr, o.Vinv, Drout, n, Np, Np);
        matmul(Vs, o.Vinv, Dsout, n, Np, Np);
    };
    build(o.rq, o.sq, o.Icub, o.Dr, o.Ds);
    // face points: face 0 (t,-1), face 1 (-t,t), face 2 (-1,-t)
    std::vector<double> fr(Nf), fs(Nf);
    for (int g = 0; g < Ng; ++g) {
        const double t = o.tg[g];
        fr[g] = t;            fs[g] = -1.0;
        fr[Ng + g] = -t;      fs[Ng + g] = t;
        fr[2 * Ng + g] = -1.0; fs[2 * Ng + g] = -t;
    }
    build(fr, fs, o.Ig, o.Drg, o.Dsg);

    // mass on T and its inverse
    o.Mref.assign((size_t)Np * Np, 0.0);
    for (int i = 0; i < Np; ++i)
        for (int j = 0; j < Np; ++j) {
            double v = 0.0;
            for (int n = 0; n < Nq; ++n) v += o.Icub[(size_t)n * Np + i] * o.wq[n] * o.Icub[(size_t)n * Np + j];
            o.Mref[(size_t)i * Np + j] = v;
        }
    o.Mrefinv.assign((size_t)Np * Np, 0.0);
    if (!spd_inverse(o.Mref.data(), o.Mrefinv.data(), Np)) {
        err = "reference mass matrix not SPD";
        return false;
    }

    o.DrW.assign((size_t)Np * Nq, 0.0);
    o.DsW.assign((size_t)Np * Nq, 0.0);
    for (int i = 0; i < Np; ++i)
        for (int n = 0; n < Nq; ++n) {
            o.DrW[(size_t)i * Nq + n] = o.Dr[(size_t)n * Np + i] * o.wq[n];
            o.DsW[(size_t)i * Nq + n] = o.Ds[(size_t)n * Np + i] * o.wq[n];
        }
    o.Lift.assign((size_t)Np * Nf, 0.0);
    for (int i = 0; i < Np; ++i)
        for (int fg = 0; fg < Nf; ++fg) o.Lift[(size_t)i * Nf + fg] = o.Ig[(size_t)fg * Np + i] * o.wg[fg % Ng];
    matmul(o.Mrefinv, o.DrW, o.MrW, Np, Np, Nq);
    matmul(o.Mrefinv, o.DsW, o.MsW, Np, Np, Nq);
    matmul(o.Mrefinv, o.Lift, o.MLift, Np, Np, Nf);
    matmul(o.MrW, o.Icub, o.Qr, Np, Nq, Np);
    matmul(o.MsW, o.Icub, o.Qs, Np, Nq, Np);

    // interpolation of the degree-N modal part to the cubature points
    std::vector<double> Ptop((size_t)Np * Np, 0.0);
    for (int m = 0; m < Np; ++m) Ptop[(size_t)m * Np + m] = (o.degree[m] == N) ? 1.0 : 0.0;
    std::vector<double> Vq((size_t)Nq * Np), tmp, tmp2;
    for (int n = 0; n < Nq; ++n)
        for (int m = 0; m < Np; ++m) psi(I[m], J[m], o.rq[n], o.sq[n], &Vq[(size_t)n * Np + m], nullptr, nullptr);
    matmul(Vq, Ptop, tmp, Nq, Np, Np);
    matmul(tmp, o.Vinv, o.Itop, Nq, Np, Np);
    return true;
}

// Prolongation between degrees (paper Sec. 5, p-refinement): the nodal
// values at the degree-Nt nodes of the degree-Nf interpolant,
// P = V_f(r_t) V_f^-1 ([Np(Nt)][Np(Nf)]).  The modal basis is hierarchical,
// so the embedded solution has zero modes of degree above Nf.
bool build_prolongation(int Nf, int Nt, std::vector<double>& P, std::string& err) {
    if (Nf < 1 || Nt < Nf) {
        err = "prolongation needs 1 <= Nf <= Nt";
        return false;
    }
    RefOps from;
    if (!build_refops(Nf, 0, from, err)) return false;
    std::vector<double> rt, st;
    nodes_2d(Nt, rt, st);
    std::vector<int> I, J;
    mode_ij(Nf, I, J);
    const int npf = n_modes(Nf), npt = (int)rt.size();
    std::vector<double> Vft((size_t)npt * npf);
    for (int k = 0; k < npt; ++k)
        for (int m = 0; m < npf; ++m) psi(I[m], J[m], rt[k], st[k], &Vft[(size_t)k * npf + m], nullptr, nullptr);
    matmul(Vft, from.Vinv, P, npt, npf, npf);
    return true;
}

}  // namespace dgc
