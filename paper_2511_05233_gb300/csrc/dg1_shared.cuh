// DG1 (tensor-product Q1) definitions shared by the kernels of dg1.cu and jvp1.cu: node and
// face-point indexing of a voxel and the pointwise node terms (storage and reaction sources).
//
// A voxel has 8 nodes on the 2-point Gauss-Legendre points, node = a + 2b + 4c for the x, y, z
// node coordinates.  In direction d the nodes form 4 lines of 2 nodes; line q meets one face
// point on either face of the voxel.  Transport factors are kept in 32 slots per voxel: the 8
// nodes, then the 24 face points (6 faces x 4 points).
#pragma once
#include "internal.h"

namespace dgls {
namespace dg1 {
constexpr double SQ3 = 1.7320508075688772935;
constexpr double ALPHA = 0.5 * (1.0 + SQ3);   // trace weight of the node next to the face
constexpr double BETA = 0.5 * (1.0 - SQ3);    // trace weight of the far node
constexpr int NG = 32;                         // g slots per voxel: 8 nodes + 6 faces x 4 points

__device__ __forceinline__ void cell_ijk(const DevParams& p, int cell, int& i, int& j, int& k) {
    i = cell % p.nx;
    int r = cell / p.nx;
    j = r % p.ny;
    k = r / p.ny;
}

// node index from per-direction node coordinates
__device__ __forceinline__ int node_of(int ax, int ay, int az) { return ax + 2 * ay + 4 * az; }

// the two nodes of line q (0..3) in direction d: n0 has coordinate 0 along d, n1 has 1
__device__ __forceinline__ void line_nodes(int d, int q, int& n0, int& n1) {
    int u = q & 1, w = q >> 1;
    if (d == 0) { n0 = node_of(0, u, w); n1 = node_of(1, u, w); }
    else if (d == 1) { n0 = node_of(u, 0, w); n1 = node_of(u, 1, w); }
    else { n0 = node_of(u, w, 0); n1 = node_of(u, w, 1); }
}

// g-slot of face (d, side) point q: 8 + (2d + (side > 0)) * 4 + q
__device__ __forceinline__ int face_slot(int d, int side, int q) { return 8 + (2 * d + (side > 0 ? 1 : 0)) * 4 + q; }

template <class S>
__device__ __forceinline__ S ld(const S* z, const DevParams& p, int f, int node, int idx) {
    return z[p.off[f] + (int64_t)node * p.flen[f] + idx];
}
}  // namespace dg1


using namespace dg1;

// Node terms of one DG1 node (mass h^3/8): storage (Eq. 50, or the relaxation's d_t Phi terms of
// Sec. 2.8) minus the reaction sources at structure points (Tab. 4).  old: the node's values at
// the previous time level (they enter only as constants).
template <class Chem, class T>
__device__ __forceinline__ void node_terms(const DevParams& p, int ph, const T* c, const T* es, T phiL, T phiS,
                                           const double* old, double tH, double dt, int relax, T* R) {
    typedef typename Base<T>::type Sc;
    constexpr int NL = Chem::NL, NS = Chem::NS, PHIL = Chem::PHIL, PHIS = Chem::PHIS;
    const bool st = ph == 1;
    const double M = p.V / 8.0;
    const Sc Mdt = Sc(M / dt);
#pragma unroll
    for (int f = 0; f < Chem::NF; ++f) R[f] = Make<T>::c(0.0);
    T epsL = liquid_fraction<Chem, T>(p, ph, es);
    double esn[2] = {0.0, 0.0};
    if (NS == 2) { esn[0] = old[NL]; esn[1] = old[NL + 1]; }
    double epsLn = val(liquid_fraction<Chem, double>(p, ph, esn));
#pragma unroll
    for (int m = 0; m < NL; ++m) {
        if (relax) R[m] = (c[m] - Make<T>::c(old[m])) * Mdt;
        else R[m] = (epsL * c[m] - Make<T>::c(epsLn * old[m])) * Mdt;
    }
    if (st) {
#pragma unroll
        for (int q = 0; q < NS; ++q) R[NL + q] = (es[q] - Make<T>::c(old[NL + q])) * Sc(M * p.rhoM[q] / dt);
    }
    if (relax) {
        R[PHIL] = (phiL - Make<T>::c(old[PHIL])) * Mdt;
        if (st) R[PHIS] = (phiS - Make<T>::c(old[PHIS])) * Mdt;
    }
    if (st) {
        T Sv[NL], Ss[2], qL, qS;
        sources<Chem, T>(p, c, es, phiL, phiS, tH, Sv, Ss, qL, qS);
        if (!relax) {
#pragma unroll
            for (int m = 0; m < NL; ++m) R[m] -= Sv[m] * Sc(M);
#pragma unroll
            for (int q = 0; q < NS; ++q) R[NL + q] -= Ss[q] * Sc(M);
        }
        R[PHIL] -= qL * Sc(M);
        R[PHIS] -= qS * Sc(M);
    }
}

}  // namespace dgls
