// Reference-tetrahedron operators of degree N, built on the host in FP64
// (paper Sec. 2 with d = 3).  The library's own implementation; it shares no
// code with the test oracle.
//
// Reference element {r, s, t >= -1, r + s + t <= -1}, vertices
// v0 = (-1,-1,-1), v1 = (1,-1,-1), v2 = (-1,1,-1), v3 = (-1,-1,1).  Face f
// has the local vertices FACE3[f] = (a, b, c), ordered so that
// (vb - va) x (vc - va) points outward; its own parametrisation is
// x(u, v) = va (-(u+v)/2) + vb (1+u)/2 + vc (1+v)/2 over the reference
// triangle.  Face-rule points live in the face's canonical frame (vertices
// by increasing global number): for orientation code o the frame's vertex m
// is the face's local vertex PERM3[o][m].
#pragma once
#include <string>
#include <vector>

namespace dgc {

extern const int FACE3[4][3];
extern const int PERM3[6][3];
extern const double VERT3[4][3];

struct RefOps3 {
    int N = 0, Np = 0, Nfp = 0, q = 0, Nq = 0, Ng = 0;
    std::vector<double> r, s, t;              // nodes [Np]
    std::vector<double> rq, sq, tq, wq;       // volume rule [Nq]
    std::vector<double> wg;                   // face rule weights [Ng] (triangle of area 2)
    std::vector<double> mu;                   // face rule frame barycentrics [Ng][3]
    std::vector<double> V, Vinv;              // [Np][Np]
    std::vector<double> Icub, Dr, Ds, Dt;     // [Nq][Np]
    std::vector<double> DrW, DsW, DtW;        // [Np][Nq]  D^T diag(W)
    std::vector<double> Mref, Mrefinv;        // [Np][Np]
    std::vector<int> fmask;                   // [4][Nfp] node of each face node (face-local lattice order)
    std::vector<int> fpos;                    // [4][Np] face-local index of a node, -1 off the face
    std::vector<double> I2;                   // [6][Ng][Nfp] face nodes -> frame points, by orientation
    std::vector<double> Dfr, Dfs, Dft;        // [4][6][Ng][Np] derivatives at the frame points
};

int n_modes3(int N);
int n_face_nodes3(int N);
bool build_refops3(int N, RefOps3& out, std::string& err);
bool build_prolongation3(int Nf, int Nt, std::vector<double>& P, std::string& err);

}  // namespace dgc
