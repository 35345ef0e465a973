// Reference-element operators of degree N, built on the host in FP64.
//
// Paper Sec. 2: orthonormal hierarchical modal basis psi_j on the reference
// triangle, collocation nodes after Warburton (warp & blend), Vandermonde
// matrix V, interpolation to cubature / face points I_cub = V_cub V^-1,
// I_g = V_g V^-1, derivative matrices D_r = V_r V^-1, D_s, mass matrix
// M = I_cub^T diag(J W) I_cub (eq. mass) and face mass I_g^T diag(W_g)
// (eq. face_mass).  This is the library's own implementation; it shares no
// code with the test oracle.
#pragma once
#include <string>
#include <vector>

namespace dgc {

struct RefOps {
    int N = 0, Np = 0, q = 0, Nq = 0, Ng = 0, Nf = 0;
    std::vector<double> r, s;          // collocation nodes [Np]
    std::vector<double> rq, sq, wq;    // volume rule [Nq]
    std::vector<double> tg, wg;        // edge rule [Ng]
    std::vector<double> V, Vinv;       // [Np][Np], V[i][j] = psi_j(r_i)
    std::vector<double> Icub, Dr, Ds;  // [Nq][Np]
    std::vector<double> Ig, Drg, Dsg;  // [3 Ng][Np], row f*Ng+g
    std::vector<double> Mref, Mrefinv; // [Np][Np] mass on T (J = 1)
    std::vector<int> degree;           // total degree of mode j
    // products used by the kernels
    std::vector<double> DrW, DsW;      // [Np][Nq]  D_r^T diag(W)
    std::vector<double> Lift;          // [Np][Nf]  I_g^T diag(w_g) over all faces
    std::vector<double> MrW, MsW, MLift;  // Mref^-1 DrW, Mref^-1 DsW, Mref^-1 Lift
    std::vector<double> Qr, Qs;        // [Np][Np]  Mref^-1 DrW I_cub, Mref^-1 DsW I_cub
    std::vector<double> Itop;          // [Nq][Np]  V_cub P_top V^-1 (degree-N modes only)
};

int default_q(int N);
int n_modes(int N);
bool build_refops(int N, int q, RefOps& out, std::string& err);
// P = V_f(r_t) V_f^-1 [Np(Nt)][Np(Nf)]: degree-Nf interpolant at the degree-Nt nodes.
bool build_prolongation(int Nf, int Nt, std::vector<double>& P, std::string& err);

// Building blocks shared with the tetrahedral operators (refops3.cpp).
namespace detail {
double jac(double x, double a, double b, int n);     // orthonormal Jacobi polynomial
double djac(double x, double a, double b, int n);    // its derivative
void gauss_jacobi(int n, double a, double b, std::vector<double>& x, std::vector<double>& w);
std::vector<double> gll(int N);                       // Gauss-Lobatto-Legendre points
void nodes_2d(int N, std::vector<double>& r, std::vector<double>& s);   // triangle warp & blend nodes
void mode_ij(int N, std::vector<int>& I, std::vector<int>& J);
void psi(int i, int j, double r, double s, double* val, double* dr, double* ds);   // triangle basis
void matmul(const std::vector<double>& A, const std::vector<double>& B, std::vector<double>& C, int n, int k,
            int m);
}  // namespace detail

// Dense helpers (row-major), used by the geometry set-up as well.
bool invert(std::vector<double>& A, int n);            // Gauss-Jordan, partial pivoting
bool spd_inverse(const double* A, double* Ainv, int n); // via Cholesky, false if not SPD

}  // namespace dgc
