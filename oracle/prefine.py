"""p-refinement (paper Sec. 5 and Table 2): a solution converged at degree
N is carried to a higher degree M by evaluating its degree-N polynomial at
the degree-M nodes in every element,

    U_M = P U_N,   P = V_N(r_M) V_N^-1   (N_p(M) x N_p(N)),

where V_N(r_M)[i][j] is the j-th degree-N mode at the i-th degree-M node.
The modal basis is hierarchical (modes ordered by total degree, the same
functions at every degree), so in the degree-M basis the embedded solution
keeps its modal coefficients of degree <= N and has zeros above.

Test infrastructure only.
"""
import numpy as np

from . import basis, nodes, tet


def prolongation(N, M):
    """P: nodal values at the degree-M nodes of a degree-N nodal field."""
    if M < N:
        raise ValueError("prolongation goes from a lower to a higher degree")
    rN, sN = nodes.warp_blend_nodes(N)
    rM, sM = nodes.warp_blend_nodes(M)
    return basis.vandermonde(N, rM, sM) @ np.linalg.inv(basis.vandermonde(N, rN, sN))


def prolong_state(U, N, M):
    """U[K][4][N_p(N)] -> [K][4][N_p(M)]."""
    return np.einsum('ij,kvj->kvi', prolongation(N, M), U)


def prolongation3(N, M):
    """The same on tetrahedra (paper Sec. 5 refines its 3D runs from p = 2
    to 3 and 4): P = V_N(r_M) V_N^-1 with the tetrahedral modes and nodes."""
    if M < N:
        raise ValueError("prolongation goes from a lower to a higher degree")
    rN, sN, tN = tet.warp_blend_nodes_3d(N)
    rM, sM, tM = tet.warp_blend_nodes_3d(M)
    return tet.vandermonde(N, rM, sM, tM) @ np.linalg.inv(tet.vandermonde(N, rN, sN, tN))


def prolong_state3(U, N, M):
    """U[K][5][N_p(N)] -> [K][5][N_p(M)]."""
    return np.einsum('ij,kvj->kvi', prolongation3(N, M), U)
