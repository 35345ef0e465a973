// Host FP64 construction of the reference-tetrahedron operators (see
// refops3.h).
#include "refops3.h"

#include <array>
#include <cmath>
#include <map>
#include <tuple>

#include "refops.h"

namespace dgc {

const int FACE3[4][3] = {{0, 2, 1}, {0, 1, 3}, {1, 2, 3}, {0, 3, 2}};
const int PERM3[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
const double VERT3[4][3] = {{-1, -1, -1}, {1, -1, -1}, {-1, 1, -1}, {-1, -1, 1}};

int n_modes3(int N) { return (N + 1) * (N + 2) * (N + 3) / 6; }
int n_face_nodes3(int N) { return (N + 1) * (N + 2) / 2; }

namespace {

using detail::djac;
using detail::jac;

// Modes by total degree, then i, then j.
void modes3(int N, std::vector<std::tuple<int, int, int>>& m) {
    m.clear();
    for (int d = 0; d <= N; ++d)
        for (int i = 0; i <= d; ++i)
            for (int j = 0; j <= d - i; ++j) m.emplace_back(i, j, d - i - j);
}

double ipow(double x, int e) { return e <= 0 ? 1.0 : std::pow(x, e); }

// psi_ijk = 2 sqrt2 P_i(a) P_j^(2i+1,0)(b) (1-b)^i P_k^(2i+2j+2,0)(c) (1-c)^(i+j)
// and its gradient; a = 2(1+r)/(-s-t) - 1, b = 2(1+s)/(1-t) - 1, c = t.
void psi3(int i, int j, int k, double r, double s, double t, double* val, double* dr, double* ds, double* dt) {
    const double den_a = -s - t, den_b = 1.0 - t;
    const double a = (std::fabs(den_a) > 1e-14) ? 2.0 * (1.0 + r) / den_a - 1.0 : -1.0;
    const double b = (std::fabs(den_b) > 1e-14) ? 2.0 * (1.0 + s) / den_b - 1.0 : -1.0;
    const double c = t;
    const double ai = 2.0 * i + 1.0, ak = 2.0 * (i + j) + 2.0;
    const double fa = jac(a, 0.0, 0.0, i), gb = jac(b, ai, 0.0, j), hc = jac(c, ak, 0.0, k);
    const double ob = 1.0 - b, oc = 1.0 - c;
    const double K = 2.0 * std::sqrt(2.0);
    if (val) *val = K * fa * gb * ipow(ob, i) * hc * ipow(oc, i + j);
    if (!dr && !ds && !dt) return;
    const double dfa = djac(a, 0.0, 0.0, i), dgb = djac(b, ai, 0.0, j), dhc = djac(c, ak, 0.0, k);
    // d/da divided by (1-b)(1-c); zero for i = 0
    const double pa = (i > 0) ? dfa * gb * ipow(ob, i - 1) * hc * ipow(oc, i + j - 1) : 0.0;
    // d/db divided by (1-c); zero for i + j = 0
    double pb = 0.0;
    if (i + j > 0) {
        double g = dgb * ipow(ob, i);
        if (i > 0) g -= i * gb * ipow(ob, i - 1);
        pb = fa * g * hc * ipow(oc, i + j - 1);
    }
    double h = dhc * ipow(oc, i + j);
    if (i + j > 0) h -= (i + j) * hc * ipow(oc, i + j - 1);
    const double pc = fa * gb * ipow(ob, i) * h;
    if (dr) *dr = K * 4.0 * pa;
    if (ds) *ds = K * (2.0 * (1.0 + a) * pa + 2.0 * pb);
    if (dt) *dt = K * (2.0 * (1.0 + a) * pa + (1.0 + b) * pb + pc);
}

// Warp & blend nodes on the tetrahedron (blending parameter 0): equidistant
// lattice on the equilateral tetrahedron, each face's triangle warp blended
// into the interior by Lb Lc Ld / ((Lb + La/2)(Lc + La/2)(Ld + La/2)), nodes
// on a face's edges taking that face's warp alone; barycentrics back to the
// reference element.  Lattice order k outer, j, i inner.
void nodes3(int N, std::vector<double>& r, std::vector<double>& s, std::vector<double>& t,
            std::vector<std::array<int, 4>>* lattice) {
    const double q3 = std::sqrt(3.0), q6 = std::sqrt(6.0);
    const double E[4][3] = {{-1.0, -1.0 / q3, -1.0 / q6}, {1.0, -1.0 / q3, -1.0 / q6},
                            {0.0, 2.0 / q3, -1.0 / q6}, {0.0, 0.0, 3.0 / q6}};
    const std::vector<double> xg = detail::gll(N);
    std::vector<double> xe(N + 1);
    for (int i = 0; i <= N; ++i) xe[i] = -1.0 + 2.0 * i / N;
    auto warp1 = [&](double x) {
        if (std::fabs(x) >= 1.0 - 1e-10) return 0.0;
        double w = 0.0;
        for (int i = 0; i <= N; ++i) {
            double l = 1.0;
            for (int m = 0; m <= N; ++m)
                if (m != i) l *= (x - xe[m]) / (xe[i] - xe[m]);
            w += (xg[i] - xe[i]) * l;
        }
        return w / (1.0 - x * x);
    };
    // barycentrics of a point of the equilateral tetrahedron
    std::vector<double> A(16);
    for (int v = 0; v < 4; ++v) {
        for (int d = 0; d < 3; ++d) A[d * 4 + v] = E[v][d];
        A[12 + v] = 1.0;
    }
    if (!invert(A, 4)) return;
    r.clear(); s.clear(); t.clear();
    if (lattice) lattice->clear();
    const double tol = 1e-10;
    for (int k = 0; k <= N; ++k)
        for (int j = 0; j <= N - k; ++j)
            for (int i = 0; i <= N - j - k; ++i) {
                const double L[4] = {1.0 - double(i + j + k) / N, double(i) / N, double(j) / N, double(k) / N};
                double X[3], S[3] = {0, 0, 0};
                for (int d = 0; d < 3; ++d) X[d] = L[0] * E[0][d] + L[1] * E[1][d] + L[2] * E[2][d] + L[3] * E[3][d];
                bool fixed = false;
                for (int fa = 0; fa < 4; ++fa) {
                    int o[3], n = 0;
                    for (int v = 0; v < 4; ++v)
                        if (v != fa) o[n++] = v;
                    double W[3] = {0, 0, 0};
                    for (int e = 0; e < 3; ++e) {
                        const int p = o[e], qv = o[(e + 1) % 3];
                        double dv[3], len = 0.0;
                        for (int d = 0; d < 3; ++d) {
                            dv[d] = E[qv][d] - E[p][d];
                            len += dv[d] * dv[d];
                        }
                        len = std::sqrt(len);
                        const double f = 4.0 * L[p] * L[qv] * warp1(L[qv] - L[p]);
                        for (int d = 0; d < 3; ++d) W[d] += f * dv[d] / len;
                    }
                    const double La = L[fa], Lb = L[o[0]], Lc = L[o[1]], Ld = L[o[2]];
                    const double den = (Lb + 0.5 * La) * (Lc + 0.5 * La) * (Ld + 0.5 * La);
                    const double blend = den > tol ? Lb * Lc * Ld / den : 0.0;
                    const int npos = (Lb > tol) + (Lc > tol) + (Ld > tol);
                    if (La < tol && npos < 3) {
                        if (!fixed)
                            for (int d = 0; d < 3; ++d) S[d] = W[d];
                        fixed = true;
                    } else if (!fixed) {
                        for (int d = 0; d < 3; ++d) S[d] += blend * W[d];
                    }
                }
                double lam[4];
                for (int v = 0; v < 4; ++v)
                    lam[v] = A[v * 4 + 0] * (X[0] + S[0]) + A[v * 4 + 1] * (X[1] + S[1]) +
                             A[v * 4 + 2] * (X[2] + S[2]) + A[v * 4 + 3];
                double P[3] = {0, 0, 0};
                for (int v = 0; v < 4; ++v)
                    for (int d = 0; d < 3; ++d) P[d] += lam[v] * VERT3[v][d];
                r.push_back(P[0]);
                s.push_back(P[1]);
                t.push_back(P[2]);
                if (lattice) lattice->push_back({N - i - j - k, i, j, k});
            }
}

}  // namespace

bool build_refops3(int N, RefOps3& o, std::string& err) {
    if (N < 1 || N > 6) {
        err = "tetrahedral degree N out of range";
        return false;
    }
    const int q = default_q(N);
    o.N = N;
    o.Np = n_modes3(N);
    o.Nfp = n_face_nodes3(N);
    o.q = q;
    o.Nq = q * q * q;
    o.Ng = q * q;
    const int Np = o.Np, Nq = o.Nq, Ng = o.Ng, Nfp = o.Nfp;
    std::vector<std::array<int, 4>> lat;
    nodes3(N, o.r, o.s, o.t, &lat);
    if ((int)o.r.size() != Np) {
        err = "tetrahedral node construction failed";
        return false;
    }
    std::vector<std::tuple<int, int, int>> M;
    modes3(N, M);
    auto vand = [&](const std::vector<double>& pr, const std::vector<double>& ps, const std::vector<double>& pt,
                    std::vector<double>* V, std::vector<double>* Vr, std::vector<double>* Vs,
                    std::vector<double>* Vt) {
        const int n = (int)pr.size();
        for (auto* X : {V, Vr, Vs, Vt})
            if (X) X->assign((size_t)n * Np, 0.0);
        for (int p = 0; p < n; ++p)
            for (int m = 0; m < Np; ++m) {
                const auto [i, j, k] = M[m];
                const size_t at = (size_t)p * Np + m;
                psi3(i, j, k, pr[p], ps[p], pt[p], V ? &(*V)[at] : nullptr, Vr ? &(*Vr)[at] : nullptr,
                     Vs ? &(*Vs)[at] : nullptr, Vt ? &(*Vt)[at] : nullptr);
            }
    };
    vand(o.r, o.s, o.t, &o.V, nullptr, nullptr, nullptr);
    o.Vinv = o.V;
    if (!invert(o.Vinv, Np)) {
        err = "singular tetrahedral Vandermonde matrix";
        return false;
    }

    // volume rule: Gauss-Legendre (a) x Gauss-Jacobi(1,0) (b) x Gauss-Jacobi(2,0) (c)
    std::vector<double> a, wa, b, wb, c, wc;
    detail::gauss_jacobi(q, 0.0, 0.0, a, wa);
    detail::gauss_jacobi(q, 1.0, 0.0, b, wb);
    detail::gauss_jacobi(q, 2.0, 0.0, c, wc);
    o.rq.resize(Nq); o.sq.resize(Nq); o.tq.resize(Nq); o.wq.resize(Nq);
    for (int kc = 0; kc < q; ++kc)
        for (int jb = 0; jb < q; ++jb)
            for (int ia = 0; ia < q; ++ia) {
                const int n = (kc * q + jb) * q + ia;
                o.rq[n] = 0.25 * (1.0 + a[ia]) * (1.0 - b[jb]) * (1.0 - c[kc]) - 1.0;
                o.sq[n] = 0.5 * (1.0 + b[jb]) * (1.0 - c[kc]) - 1.0;
                o.tq[n] = c[kc];
                o.wq[n] = wa[ia] * wb[jb] * wc[kc] / 8.0;
            }
    std::vector<double> Vq, Vr, Vs, Vt;
    vand(o.rq, o.sq, o.tq, &Vq, &Vr, &Vs, &Vt);
    detail::matmul(Vq, o.Vinv, o.Icub, Nq, Np, Np);
    detail::matmul(Vr, o.Vinv, o.Dr, Nq, Np, Np);
    detail::matmul(Vs, o.Vinv, o.Ds, Nq, Np, Np);
    detail::matmul(Vt, o.Vinv, o.Dt, Nq, Np, Np);

    // face rule: the triangle's collapsed rule in the frame's coordinates
    o.wg.resize(Ng);
    o.mu.resize((size_t)Ng * 3);
    for (int jb = 0; jb < q; ++jb)
        for (int ia = 0; ia < q; ++ia) {
            const int g = jb * q + ia;
            const double u = 0.5 * (1.0 + a[ia]) * (1.0 - b[jb]) - 1.0, v = b[jb];
            o.wg[g] = 0.5 * wa[ia] * wb[jb];
            o.mu[3 * g] = -(u + v) / 2.0;
            o.mu[3 * g + 1] = (1.0 + u) / 2.0;
            o.mu[3 * g + 2] = (1.0 + v) / 2.0;
        }

    // face nodes in face-local lattice order (j outer, i inner) from the
    // lattice counts of the vertices
    std::map<std::array<int, 4>, int> at;
    for (int n = 0; n < Np; ++n) at[lat[n]] = n;
    o.fmask.assign((size_t)4 * Nfp, -1);
    o.fpos.assign((size_t)4 * Np, -1);
    for (int f = 0; f < 4; ++f) {
        int n = 0;
        for (int j = 0; j <= N; ++j)
            for (int i = 0; i <= N - j; ++i, ++n) {
                std::array<int, 4> cnt = {0, 0, 0, 0};
                cnt[FACE3[f][0]] = N - i - j;
                cnt[FACE3[f][1]] = i;
                cnt[FACE3[f][2]] = j;
                const auto it = at.find(cnt);
                if (it == at.end()) {
                    err = "face node not found";
                    return false;
                }
                o.fmask[(size_t)f * Nfp + n] = it->second;
                o.fpos[(size_t)f * Np + it->second] = n;
            }
    }
    // 2D Vandermonde of the face nodes in face-local (u, v) (the same for all
    // faces: the face-local lattice order follows each face's own vertices)
    std::vector<int> I2m, J2m;
    detail::mode_ij(N, I2m, J2m);
    auto face_uv = [&](int node, int f, double& u, double& v) {
        const double lam[4] = {-(1.0 + o.r[node] + o.s[node] + o.t[node]) / 2.0, (1.0 + o.r[node]) / 2.0,
                               (1.0 + o.s[node]) / 2.0, (1.0 + o.t[node]) / 2.0};
        u = 2.0 * lam[FACE3[f][1]] - 1.0;
        v = 2.0 * lam[FACE3[f][2]] - 1.0;
    };
    for (int f = 1; f < 4; ++f)
        for (int n = 0; n < Nfp; ++n) {
            double u0, v0, u, v;
            face_uv(o.fmask[n], 0, u0, v0);
            face_uv(o.fmask[(size_t)f * Nfp + n], f, u, v);
            if (std::fabs(u - u0) > 1e-12 || std::fabs(v - v0) > 1e-12) {
                err = "face node sets differ between faces";
                return false;
            }
        }
    std::vector<double> V2((size_t)Nfp * Nfp);
    for (int n = 0; n < Nfp; ++n) {
        double u, v;
        face_uv(o.fmask[n], 0, u, v);
        for (int m = 0; m < Nfp; ++m) detail::psi(I2m[m], J2m[m], u, v, &V2[(size_t)n * Nfp + m], nullptr, nullptr);
    }
    if (!invert(V2, Nfp)) {
        err = "singular face Vandermonde matrix";
        return false;
    }
    o.I2.assign((size_t)6 * Ng * Nfp, 0.0);
    o.Dfr.assign((size_t)24 * Ng * Np, 0.0);
    o.Dfs = o.Dfr;
    o.Dft = o.Dfr;
    for (int ori = 0; ori < 6; ++ori) {
        std::vector<double> Vp((size_t)Ng * Nfp), prod;
        for (int g = 0; g < Ng; ++g) {
            double lam[3];
            for (int m = 0; m < 3; ++m) lam[PERM3[ori][m]] = o.mu[3 * g + m];
            const double u = 2.0 * lam[1] - 1.0, v = 2.0 * lam[2] - 1.0;
            for (int m = 0; m < Nfp; ++m) detail::psi(I2m[m], J2m[m], u, v, &Vp[(size_t)g * Nfp + m], nullptr, nullptr);
        }
        detail::matmul(Vp, V2, prod, Ng, Nfp, Nfp);
        std::copy(prod.begin(), prod.end(), o.I2.begin() + (size_t)ori * Ng * Nfp);
        for (int f = 0; f < 4; ++f) {
            std::vector<double> pr(Ng), ps(Ng), pt(Ng);
            for (int g = 0; g < Ng; ++g) {
                double P[3] = {0, 0, 0};
                for (int m = 0; m < 3; ++m) {
                    const int vtx = FACE3[f][PERM3[ori][m]];
                    for (int d = 0; d < 3; ++d) P[d] += o.mu[3 * g + m] * VERT3[vtx][d];
                }
                pr[g] = P[0]; ps[g] = P[1]; pt[g] = P[2];
            }
            std::vector<double> Gr, Gs, Gt, Dr_, Ds_, Dt_;
            vand(pr, ps, pt, nullptr, &Gr, &Gs, &Gt);
            detail::matmul(Gr, o.Vinv, Dr_, Ng, Np, Np);
            detail::matmul(Gs, o.Vinv, Ds_, Ng, Np, Np);
            detail::matmul(Gt, o.Vinv, Dt_, Ng, Np, Np);
            const size_t off = (size_t)(f * 6 + ori) * Ng * Np;
            std::copy(Dr_.begin(), Dr_.end(), o.Dfr.begin() + off);
            std::copy(Ds_.begin(), Ds_.end(), o.Dfs.begin() + off);
            std::copy(Dt_.begin(), Dt_.end(), o.Dft.begin() + off);
        }
    }

    // reference mass and the weighted transposed derivatives
    o.Mref.assign((size_t)Np * Np, 0.0);
    for (int i = 0; i < Np; ++i)
        for (int j = 0; j < Np; ++j) {
            double v = 0.0;
            for (int n = 0; n < Nq; ++n) v += o.Icub[(size_t)n * Np + i] * o.wq[n] * o.Icub[(size_t)n * Np + j];
            o.Mref[(size_t)i * Np + j] = v;
        }
    o.Mrefinv.assign((size_t)Np * Np, 0.0);
    if (!spd_inverse(o.Mref.data(), o.Mrefinv.data(), Np)) {
        err = "reference tetrahedral mass matrix not SPD";
        return false;
    }
    o.DrW.assign((size_t)Np * Nq, 0.0);
    o.DsW = o.DrW;
    o.DtW = o.DrW;
    for (int i = 0; i < Np; ++i)
        for (int n = 0; n < Nq; ++n) {
            o.DrW[(size_t)i * Nq + n] = o.Dr[(size_t)n * Np + i] * o.wq[n];
            o.DsW[(size_t)i * Nq + n] = o.Ds[(size_t)n * Np + i] * o.wq[n];
            o.DtW[(size_t)i * Nq + n] = o.Dt[(size_t)n * Np + i] * o.wq[n];
        }
    return true;
}

// Prolongation between tetrahedral degrees (paper Sec. 5, p-refinement):
// the nodal values at the degree-Nt nodes of the degree-Nf interpolant,
// P = V_f(r_t) V_f^-1 ([Np(Nt)][Np(Nf)]); the modes are hierarchical, so
// the embedded field has no modes of degree above Nf.
bool build_prolongation3(int Nf, int Nt, std::vector<double>& P, std::string& err) {
    if (Nf < 1 || Nt < Nf) {
        err = "prolongation needs 1 <= Nf <= Nt";
        return false;
    }
    RefOps3 from;
    if (!build_refops3(Nf, from, err)) return false;
    std::vector<double> rt, st, tt;
    nodes3(Nt, rt, st, tt, nullptr);
    std::vector<std::tuple<int, int, int>> M;
    modes3(Nf, M);
    const int npf = (int)M.size(), npt = (int)rt.size();
    std::vector<double> Vft((size_t)npt * npf);
    for (int k = 0; k < npt; ++k)
        for (int m = 0; m < npf; ++m)
            psi3(std::get<0>(M[m]), std::get<1>(M[m]), std::get<2>(M[m]), rt[k], st[k], tt[k],
                 &Vft[(size_t)k * npf + m], nullptr, nullptr, nullptr);
    detail::matmul(Vft, from.Vinv, P, npt, npf, npf);
    return true;
}

}  // namespace dgc
