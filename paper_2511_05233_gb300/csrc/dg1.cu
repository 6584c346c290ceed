// DG1 (tensor-product Q1) residual, Jacobian-vector product and per-node diagonal blocks.
//
// Discretisation (Eqs. 43-47): Lagrange basis on the 2-point Gauss-Legendre nodes of each voxel,
// the same points for volume quadrature (diagonal mass h^3/8 per node) and 2 x 2 Gauss points
// per face lying on the nodal lines; interior faces carry
//   -int {K}_H {d_n psi} [[v]] + penalty int {K}_H [[psi]].[[v]] / h
// per (coefficient x gradient) term of Tab. 4, the coefficient taken from the traced fields on
// each side.  Everything factorises along nodal lines: in direction d a voxel has 4 lines of
// 2 nodes, each line meets one face point on either side, and the volume term of a line is
// +-(3h/8)(K_0 + K_1)(psi_1 - psi_0).
//
// Kernels: (A) transport factors g at the 8 nodes and the 24 face points of every voxel (the
// only exponentials of the transport part), (B1) one thread per (node, voxel) for storage and
// reaction sources, (B2) one pass per direction with one thread per (line, voxel) adding the
// volume and face terms of that line into its two nodes.  Each direction pass touches disjoint
// node pairs, so the read-modify-write of B2 is race free without atomics.
#include "dg1_shared.cuh"

namespace dgls {

static inline int nblocks(int64_t n, int bs) { return (int)((n + bs - 1) / bs); }

// ------------------------------------------------------------------ (A) transport factors
template <class Chem, class S, bool TAN>
__global__ void __launch_bounds__(128) k_dg1_g(const DevParams p, const Geo g, const S* __restrict__ z,
                                               const S* __restrict__ v, S* __restrict__ gb, S* __restrict__ gbd) {
    int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= p.n_cell) return;
    typedef typename std::conditional<TAN, Dual<S>, S>::type T;
    constexpr int NL = Chem::NL, NS = Chem::NS;
    const int ph = g.phase[cell];
    const int s = g.cmap[cell];
    // nodal concentrations and solid fractions
    T c[8][NL], es[8][2];
#pragma unroll
    for (int n = 0; n < 8; ++n) {
#pragma unroll
        for (int m = 0; m < NL; ++m)
            c[n][m] = Make<T>::var(ld(z, p, m, n, cell), TAN ? (double)ld(v, p, m, n, cell) : 0.0);
        es[n][0] = es[n][1] = Make<T>::c(0.0);
        if (NS == 2 && ph == 1) {
#pragma unroll
            for (int q = 0; q < 2; ++q)
                es[n][q] = Make<T>::var(ld(z, p, NL + q, n, s), TAN ? (double)ld(v, p, NL + q, n, s) : 0.0);
        }
        T eL = liquid_fraction<Chem, T>(p, ph, es[n]);
        T gg = transport_factor<Chem, T>(p, eL, c[n]);
        gb[(int64_t)n * p.n_cell + cell] = val(gg);
        if constexpr (TAN) gbd[(int64_t)n * p.n_cell + cell] = gg.d;
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
#pragma unroll
        for (int side = -1; side <= 1; side += 2) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                int n0, n1;
                line_nodes(d, q, n0, n1);
                const typename Base<T>::type wn = side > 0 ? ALPHA : BETA, wf = side > 0 ? BETA : ALPHA;
                T ct[NL], et[2];
#pragma unroll
                for (int m = 0; m < NL; ++m) ct[m] = c[n1][m] * wn + c[n0][m] * wf;
                et[0] = es[n1][0] * wn + es[n0][0] * wf;
                et[1] = es[n1][1] * wn + es[n0][1] * wf;
                T eL = liquid_fraction<Chem, T>(p, ph, et);
                T gg = transport_factor<Chem, T>(p, eL, ct);
                int slot = face_slot(d, side, q);
                gb[(int64_t)slot * p.n_cell + cell] = val(gg);
                if constexpr (TAN) gbd[(int64_t)slot * p.n_cell + cell] = gg.d;
            }
        }
    }
}

template <class Chem, class S, int MODE>   // MODE 0: residual (S = double), 1: JVP tangent
__global__ void __launch_bounds__(128) k_dg1_nodes(const DevParams p, const Geo g, const S* __restrict__ z,
                                                   const S* __restrict__ v, const double* __restrict__ zn,
                                                   double t, double dt, int relax, double sc_dt, S* __restrict__ r) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= (int64_t)p.n_cell * 8) return;
    typedef typename std::conditional<MODE == 1, Dual<S>, S>::type T;
    constexpr int NL = Chem::NL, NS = Chem::NS, NF = Chem::NF, PHIL = Chem::PHIL, PHIS = Chem::PHIS;
    const int n = (int)(b / p.n_cell);
    const int cell = (int)(b - (int64_t)n * p.n_cell);
    const int ph = g.phase[cell];
    const int s = g.cmap[cell];
    const bool st = ph == 1;
    T c[NL], es[2], phiL, phiS;
#pragma unroll
    for (int m = 0; m < NL; ++m) c[m] = Make<T>::var(ld(z, p, m, n, cell), MODE == 1 ? (double)ld(v, p, m, n, cell) : 0.0);
    es[0] = es[1] = Make<T>::c(0.0);
    phiS = Make<T>::c(0.0);
    phiL = Make<T>::var(ld(z, p, PHIL, n, cell), MODE == 1 ? (double)ld(v, p, PHIL, n, cell) : 0.0);
    if (st) {
#pragma unroll
        for (int q = 0; q < NS; ++q) es[q] = Make<T>::var(ld(z, p, NL + q, n, s), MODE == 1 ? (double)ld(v, p, NL + q, n, s) : 0.0);
        phiS = Make<T>::var(ld(z, p, PHIS, n, s), MODE == 1 ? (double)ld(v, p, PHIS, n, s) : 0.0);
    }
    double old[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        old[f] = 0.0;
        if (MODE == 0) {
            if (!p.is_struct[f]) old[f] = zn[p.off[f] + (int64_t)n * p.flen[f] + cell];
            else if (st) old[f] = zn[p.off[f] + (int64_t)n * p.flen[f] + s];
        }
    }
    T R[NF];
    node_terms<Chem, T>(p, ph, c, es, phiL, phiS, old, smooth_step(t), dt, relax, R);
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        if (p.is_struct[f] && !st) continue;
        int64_t o = p.off[f] + (int64_t)n * p.flen[f] + (p.is_struct[f] ? s : cell);
        if constexpr (MODE == 1) {
            S val_ = R[f].d;
            if (sc_dt > 0.0) val_ = val_ * S(sc_dt * p.rscale[f]);
            r[o] = val_;
        } else {
            r[o] = R[f];
        }
    }
}

// ------------------------------------------------------------------ (B2) lines: volume + faces
// Dual-number form, launched where no linearisation is current (the public dg_jvp of a
// mixed-precision context): one thread per (line, voxel) of direction d, evaluating both faces of
// its line.
// The fields are streamed one at a time (register pressure: the whole line with both neighbours
// would hold ~100 dual numbers), each field's two nodal outputs are read-modify-written as soon as
// they are complete.
template <class Chem, class S, int MODE>    // MODE 1: JVP tangent (the residual uses k_res_face/gather)
__global__ void __launch_bounds__(128) k_dg1_lines(const DevParams p, const Geo g, const S* __restrict__ z,
                                                   const S* __restrict__ v, const S* __restrict__ gb,
                                                   const S* __restrict__ gbd, int d, double t, double dt, int relax,
                                                   double sc_dt, S* __restrict__ r) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= (int64_t)p.n_cell * 4) return;
    typedef typename std::conditional<MODE == 1, Dual<S>, S>::type T;
    typedef S Sc;
    constexpr int NL = Chem::NL;
    const bool tan = MODE == 1;
    const int q = (int)(b / p.n_cell);
    const int cell = (int)(b - (int64_t)q * p.n_cell);
    int i, j, k;
    cell_ijk(p, cell, i, j, k);
    int n0, n1;
    line_nodes(d, q, n0, n1);
    const int ph = g.phase[cell];
    const int sidx = g.cmap[cell];
    const bool st = ph == 1;
    const Sc vol = Sc(3.0 * p.h / 8.0);
    const Sc wf = Sc(0.25 * p.h * p.h);
    const Sc gq = Sc(SQ3 / p.h);
    const Sc pen = Sc(p.penalty / p.h);
    const Sc al = Sc(ALPHA), be = Sc(BETA);

    auto gload = [&](int slot, int c) -> T {
        int64_t o = (int64_t)slot * p.n_cell + c;
        return Make<T>::var(gb[o], tan ? (double)gbd[o] : 0.0);
    };
    auto fld = [&](int f, int n, int idx) -> T {
        int64_t o = p.off[f] + (int64_t)n * p.flen[f] + idx;
        return Make<T>::var(z[o], tan ? (double)v[o] : 0.0);
    };
    // neighbours along d: side 0 = xi = -1 face (left), side 1 = xi = +1 face (right)
    const int coord = d == 0 ? i : d == 1 ? j : k;
    const int ext = d == 0 ? p.nx : d == 1 ? p.ny : p.nz;
    const int stride = d == 0 ? 1 : d == 1 ? p.nx : p.nx * p.ny;
    bool hasQ[2], stQ[2];
    int qcell[2], qsidx[2];
#pragma unroll
    for (int sd = 0; sd < 2; ++sd) {
        int qc = coord + (sd == 0 ? -1 : 1);
        hasQ[sd] = qc >= 0 && qc < ext;
        qcell[sd] = hasQ[sd] ? cell + (sd == 0 ? -stride : stride) : cell;
        stQ[sd] = hasQ[sd] && g.phase[qcell[sd]] == 1;
        qsidx[sd] = hasQ[sd] ? g.cmap[qcell[sd]] : -1;
    }
    // transport factors: nodes, own face points, neighbour face points; face harmonic means
    const T gN0 = gload(n0, cell), gN1 = gload(n1, cell);
    const T gsum = gN0 + gN1;
    T gl[2], gr[2], Hg[2];
#pragma unroll
    for (int sd = 0; sd < 2; ++sd) {
        Hg[sd] = Make<T>::c(0.0);
        gl[sd] = gr[sd] = Make<T>::c(0.0);
        if (!hasQ[sd]) continue;
        T gP = gload(face_slot(d, sd == 0 ? -1 : +1, q), cell);
        T gQ = gload(face_slot(d, sd == 0 ? +1 : -1, q), qcell[sd]);
        gl[sd] = sd == 1 ? gP : gQ;
        gr[sd] = sd == 1 ? gQ : gP;
        Hg[sd] = harm(gl[sd], gr[sd]);
    }
    // liquid potential along the line: volume difference, face jumps (left minus right) and mean
    // normal gradients
    const T PL0 = fld(Chem::PHIL, n0, cell), PL1 = fld(Chem::PHIL, n1, cell);
    const T dPhi = PL1 - PL0;
    T jL[2], mL[2];
#pragma unroll
    for (int sd = 0; sd < 2; ++sd) {
        jL[sd] = mL[sd] = Make<T>::c(0.0);
        if (!hasQ[sd]) continue;
        T Q0 = fld(Chem::PHIL, n0, qcell[sd]), Q1 = fld(Chem::PHIL, n1, qcell[sd]);
        T tP = sd == 1 ? PL1 * al + PL0 * be : PL0 * al + PL1 * be;     // own trace at this face
        T tN = sd == 1 ? Q0 * al + Q1 * be : Q1 * al + Q0 * be;         // neighbour trace
        jL[sd] = sd == 1 ? tP - tN : tN - tP;
        mL[sd] = (dPhi + (Q1 - Q0)) * (gq * Sc(0.5));
    }
    T accL0 = Make<T>::c(0.0), accL1 = Make<T>::c(0.0);
    auto add_face = [&](int sd, T f, T& a0, T& a1) {
        // left cell gets +f v-, right cell -f v+; the own near node is index sd
        T ff = f * (sd == 1 ? wf : -wf);
        if (sd == 1) { a1 += ff * al; a0 += ff * be; }
        else { a0 += ff * al; a1 += ff * be; }
    };
    auto store = [&](int f, int idx, T a0, T a1) {
        int64_t o0 = p.off[f] + (int64_t)n0 * p.flen[f] + idx;
        int64_t o1 = p.off[f] + (int64_t)n1 * p.flen[f] + idx;
        if constexpr (MODE == 1) {
            S s0 = a0.d, s1 = a1.d;
            if (sc_dt > 0.0) { S sc = S(sc_dt * p.rscale[f]); s0 *= sc; s1 *= sc; }
            r[o0] += s0;
            r[o1] += s1;
        } else {
            r[o0] += a0;
            r[o1] += a1;
        }
    };
#pragma unroll 1
    for (int m = 0; m < NL; ++m) {
        const bool charged = p.zc[m] != 0.0;
        const T C0 = fld(m, n0, cell), C1 = fld(m, n1, cell);
        const T dc = C1 - C0;
        T a0 = Make<T>::c(0.0), a1 = Make<T>::c(0.0);
        // volume term of the line
        {
            T fl = Make<T>::c(0.0);
            if (!relax) fl = gsum * dc * Sc(p.D0[m]);
            if (charged) {
                T msum = gN0 * C0 + gN1 * C1;
                if (!relax) fl += msum * dPhi * Sc(p.kappa_m[m]);
                T fL = (gsum * dc * Sc(p.Kd[m]) + msum * dPhi * Sc(p.Km[m])) * vol;
                accL1 += fL;
                accL0 -= fL;
            }
            fl = fl * vol;
            a1 += fl;
            a0 -= fl;
        }
        // faces
#pragma unroll
        for (int sd = 0; sd < 2; ++sd) {
            if (!hasQ[sd]) continue;
            T Q0 = fld(m, n0, qcell[sd]), Q1 = fld(m, n1, qcell[sd]);
            T tP = sd == 1 ? C1 * al + C0 * be : C0 * al + C1 * be;
            T tN = sd == 1 ? Q0 * al + Q1 * be : Q1 * al + Q0 * be;
            T jc = sd == 1 ? tP - tN : tN - tP;
            T mc = (dc + (Q1 - Q0)) * (gq * Sc(0.5));
            T dterm = (jc * pen - mc) * Hg[sd];
            T f = Make<T>::c(0.0);
            if (!relax) f = dterm * Sc(p.D0[m]);
            if (charged) {
                T cl = sd == 1 ? tP : tN;
                T cr = sd == 1 ? tN : tP;
                T Hm = harm(gl[sd] * cl, gr[sd] * cr);
                T mterm = (jL[sd] * pen - mL[sd]) * Hm;
                if (!relax) f += mterm * Sc(p.kappa_m[m]);
                add_face(sd, dterm * Sc(p.Kd[m]) + mterm * Sc(p.Km[m]), accL0, accL1);
            }
            add_face(sd, f, a0, a1);
        }
        // anode exchange on the x = nx face (Li+ row and, below, the Phi^L row)
        if (m == 0 && d == 0 && i == p.nx - 1) {
            T cLi = C1 * al + C0 * be;
            T phL = PL1 * al + PL0 * be;
            T rA = anode_rate<T>(p, cLi, phL);
            if (!relax) {
                T fLi = rA * (wf * Sc(p.kAno));
                a1 += fLi * al;
                a0 += fLi * be;
            }
            T fL = rA * (wf * Sc(p.F * p.kAno));
            accL1 += fL * al;
            accL0 += fL * be;
        }
        store(m, cell, a0, a1);
    }
    store(Chem::PHIL, cell, accL0, accL1);
    // solid potential (structure voxels only)
    if (st) {
        const T S0 = fld(Chem::PHIS, n0, sidx), S1 = fld(Chem::PHIS, n1, sidx);
        T a0 = Make<T>::c(0.0), a1 = Make<T>::c(0.0);
        T fs = (S1 - S0) * (Sc(2.0 * p.kappa_s) * vol);
        a1 += fs;
        a0 -= fs;
#pragma unroll
        for (int sd = 0; sd < 2; ++sd) {
            if (!hasQ[sd] || !stQ[sd]) continue;
            T Q0 = fld(Chem::PHIS, n0, qsidx[sd]), Q1 = fld(Chem::PHIS, n1, qsidx[sd]);
            T tP = sd == 1 ? S1 * al + S0 * be : S0 * al + S1 * be;
            T tN = sd == 1 ? Q0 * al + Q1 * be : Q1 * al + Q0 * be;
            T jS = sd == 1 ? tP - tN : tN - tP;
            T mS = ((S1 - S0) + (Q1 - Q0)) * (gq * Sc(0.5));
            add_face(sd, (jS * pen - mS) * Sc(p.kappa_s), a0, a1);
        }
        if (d == 0 && i == 0) {
            double fj = 0.25 * p.h * p.h * p.j_cc * (relax ? smooth_step(t) : 1.0);
            a0 += Make<T>::c(fj * ALPHA);
            a1 += Make<T>::c(fj * BETA);
        }
        store(Chem::PHIS, sidx, a0, a1);
    }
}


// ------------------------------------------------------------------ linearised FP64 JVP
// The FP64 JVP above recomputes, for every Krylov vector, the values and all transcendentals and
// divisions along with the tangents; on GB300 that keeps the FP64 pipe ~85 % busy while HBM idles.
// During one Newton iteration the linearisation point z is fixed, so the value side is computed
// once and cached (HBM is cheap here, FP64 issue is not):
//   jn   [8 nodes][NF x NF][structure voxel]  derivative of the node terms (storage + sources)
//                                    w.r.t. the node's own unknowns (pore and separator voxels:
//                                    the storage diagonal, computed where it is needed);
//   gam  [32 slots][voxel]          dg = g (gam d eps_L - visc d c_S): gam = 3/(2 eps_L) or 0;
//   face [3 dirs x 4 lines][NFD][voxel] for the +d face of each voxel: {g}_H and its two partial
//        derivatives, the flux brackets (pen [[psi]] - {d_n psi}) of every liquid field and of
//        Phi^L, and per charged species {g c}_H with the coefficients of its differential;
//        on the x = nx face: d r_Ano / d c_Li, d r_Ano / d Phi^L.
// The apply kernels are then products of cached coefficients with tangents (FMAs only).
template <class Chem>
struct LinShape {
    static constexpr int NL = Chem::NL;
    static constexpr int NC = Chem::NL - 1;                  // charged species (all but S8(L))
    static constexpr int NFD = 3 + NL + 1 + 5 * NC;
    static __device__ __forceinline__ int ci(int m) { return m < 1 ? m : m - 1; }
};

template <class Chem, class S>
__global__ void __launch_bounds__(128) k_lin_gam(const DevParams p, const Geo g, const S* __restrict__ z,
                                                 S* __restrict__ gam) {
    int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= p.n_cell) return;
    constexpr int NS = Chem::NS;
    const int ph = g.phase[cell];
    const int s = g.cmap[cell];
    S es[8][2];
#pragma unroll
    for (int n = 0; n < 8; ++n) {
        es[n][0] = es[n][1] = S(0);
        if (NS == 2 && ph == 1) {
            es[n][0] = ld(z, p, Chem::NL, n, s);
            es[n][1] = ld(z, p, Chem::NL + 1, n, s);
        }
        S eL = liquid_fraction<Chem, S>(p, ph, es[n]);
        gam[(int64_t)n * p.n_cell + cell] = (ph == 1 && NS == 2 && eL > S(0)) ? S(1.5) / eL : S(0);
    }
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int side = -1; side <= 1; side += 2)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                int n0, n1;
                line_nodes(d, q, n0, n1);
                const S wn = side > 0 ? S(ALPHA) : S(BETA), wf = side > 0 ? S(BETA) : S(ALPHA);
                S et[2] = {es[n1][0] * wn + es[n0][0] * wf, es[n1][1] * wn + es[n0][1] * wf};
                S eL = liquid_fraction<Chem, S>(p, ph, et);
                gam[(int64_t)face_slot(d, side, q) * p.n_cell + cell] = (ph == 1 && NS == 2 && eL > S(0)) ? S(1.5) / eL : S(0);
            }
}

// node Jacobians of the structure voxels: one thread per (node, structure voxel), NF seeded
// evaluations of the node terms.  Elsewhere (pore, separator) the node terms are the storage terms
// alone and their Jacobian is the diagonal that make_node_diag gives, so nothing is stored there.
template <class Chem, class S>
__global__ void __launch_bounds__(64) k_lin_nodes_build(const DevParams p, const Geo g, const S* __restrict__ z,
                                                        double t, double dt, int relax, S* __restrict__ jn) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= (int64_t)p.n_struct * 8) return;
    typedef Dual<S> T;
    constexpr int NL = Chem::NL, NS = Chem::NS, NF = Chem::NF, PHIL = Chem::PHIL, PHIS = Chem::PHIS;
    const int n = (int)(b / p.n_struct);
    const int sidx = (int)(b - (int64_t)n * p.n_struct);
    const int cell = g.sidx[sidx];
    double old[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) old[f] = 0.0;
    const double tH = smooth_step(t);
    S* J = jn + (int64_t)n * NF * NF * p.n_struct + sidx;    // [row*NF + col][structure voxel]
#pragma unroll 1
    for (int col = 0; col < NF; ++col) {
        T c[NL], es[2], phiL, phiS;
#pragma unroll
        for (int m = 0; m < NL; ++m) c[m] = Make<T>::var(ld(z, p, m, n, cell), col == m ? 1.0 : 0.0);
        phiL = Make<T>::var(ld(z, p, PHIL, n, cell), col == PHIL ? 1.0 : 0.0);
        es[0] = es[1] = Make<T>::c(0.0);
#pragma unroll
        for (int q = 0; q < NS; ++q) es[q] = Make<T>::var(ld(z, p, NL + q, n, sidx), col == NL + q ? 1.0 : 0.0);
        phiS = Make<T>::var(ld(z, p, PHIS, n, sidx), col == PHIS ? 1.0 : 0.0);
        T R[NF];
        node_terms<Chem, T>(p, 1, c, es, phiL, phiS, old, tH, dt, relax, R);
#pragma unroll
        for (int row = 0; row < NF; ++row) J[(int64_t)(row * NF + col) * p.n_struct] = R[row].d;
    }
}

// Diagonal node Jacobian of a pore or separator voxel (node terms without sources):
// d R_m / d c_m = eps_L M / dt (M / dt while relaxing) and d R_PhiL / d Phi^L = M / dt while
// relaxing, 0 otherwise.  Computed on the host once per call (no FP64 division per thread).
struct NodeDiag {
    double c_pore, c_sep, phi;
};

static NodeDiag make_node_diag(const DevParams& p, double dt, int relax) {
    const double Mdt = (p.V / 8.0) / dt;
    NodeDiag nd;
    nd.c_pore = relax ? Mdt : 1.0 * Mdt;
    nd.c_sep = relax ? Mdt : p.eps_sep * Mdt;
    nd.phi = relax ? Mdt : 0.0;
    return nd;
}

// face data of the +d face of every voxel (and the anode derivatives on the x = nx face)
template <class Chem, class S>
__global__ void __launch_bounds__(128) k_lin_faces_build(const DevParams p, const Geo g, const S* __restrict__ z,
                                                         const S* __restrict__ gb, int d, S* __restrict__ face) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= (int64_t)p.n_cell * 4) return;
    typedef LinShape<Chem> SH;
    constexpr int NL = Chem::NL;
    const int q = (int)(b / p.n_cell);
    const int cell = (int)(b - (int64_t)q * p.n_cell);
    int i, j, k;
    cell_ijk(p, cell, i, j, k);
    int n0, n1;
    line_nodes(d, q, n0, n1);
    S* F = face + (int64_t)((d * 4 + q) * SH::NFD) * p.n_cell + cell;
    auto put = [&](int kk, S v) { F[(int64_t)kk * p.n_cell] = v; };
    const int coord = d == 0 ? i : d == 1 ? j : k;
    const int ext = d == 0 ? p.nx : d == 1 ? p.ny : p.nz;
    const int stride = d == 0 ? 1 : d == 1 ? p.nx : p.nx * p.ny;
    const S pen = S(p.penalty / p.h), gq = S(SQ3 / p.h);
    if (coord + 1 >= ext) {
        if (d == 0) {   // anode face of the last layer: r_Ano derivatives at the face point
            S cLi = S(ALPHA) * ld(z, p, 0, n1, cell) + S(BETA) * ld(z, p, 0, n0, cell);
            S phL = S(ALPHA) * ld(z, p, Chem::PHIL, n1, cell) + S(BETA) * ld(z, p, Chem::PHIL, n0, cell);
            Dual<S> r1 = anode_rate<Dual<S>>(p, mkd(cLi, S(1)), mkd(phL, S(0)));
            Dual<S> r2 = anode_rate<Dual<S>>(p, mkd(cLi, S(0)), mkd(phL, S(1)));
            put(0, r1.d);
            put(1, r2.d);
        }
        return;
    }
    const int qc = cell + stride;
    const S gl = gb[(int64_t)face_slot(d, +1, q) * p.n_cell + cell];
    const S gr = gb[(int64_t)face_slot(d, -1, q) * p.n_cell + qc];
    S Hg = S(0), Ha = S(0), Hb = S(0);
    if (gl * gr > S(0)) {
        S r = S(1) / (gl + gr);
        Hg = S(2) * gl * gr * r;
        Ha = S(2) * gr * gr * r * r;
        Hb = S(2) * gl * gl * r * r;
    }
    put(0, Hg);
    put(1, Ha);
    put(2, Hb);
    {
        S P0 = ld(z, p, Chem::PHIL, n0, cell), P1 = ld(z, p, Chem::PHIL, n1, cell);
        S Q0 = ld(z, p, Chem::PHIL, n0, qc), Q1 = ld(z, p, Chem::PHIL, n1, qc);
        S jL = (S(ALPHA) * P1 + S(BETA) * P0) - (S(ALPHA) * Q0 + S(BETA) * Q1);
        S mL = S(0.5) * gq * ((P1 - P0) + (Q1 - Q0));
        put(3 + NL, jL * pen - mL);
    }
#pragma unroll
    for (int m = 0; m < NL; ++m) {
        S C0 = ld(z, p, m, n0, cell), C1 = ld(z, p, m, n1, cell);
        S Q0 = ld(z, p, m, n0, qc), Q1 = ld(z, p, m, n1, qc);
        S cl = S(ALPHA) * C1 + S(BETA) * C0, cr = S(ALPHA) * Q0 + S(BETA) * Q1;
        put(3 + m, (cl - cr) * pen - S(0.5) * gq * ((C1 - C0) + (Q1 - Q0)));
        if (p.zc[m] != 0.0) {
            const int base = 4 + NL + 5 * SH::ci(m);
            S x = gl * cl, y = gr * cr;
            S Hm = S(0), Hx = S(0), Hy = S(0);
            if (x * y > S(0)) {
                S r = S(1) / (x + y);
                Hm = S(2) * x * y * r;
                Hx = S(2) * y * y * r * r;
                Hy = S(2) * x * x * r * r;
            }
            put(base + 0, Hm);
            put(base + 1, Hx * cl);     // coefficient of d g_l
            put(base + 2, Hx * gl);     // coefficient of d c_l
            put(base + 3, Hy * cr);     // coefficient of d g_r
            put(base + 4, Hy * gr);     // coefficient of d c_r
        }
    }
}

// Per-call constants of the linearised apply, in the arithmetic type S of the product, with the
// area / volume weights and the row scales (sc_dt * rscale, or 1 for the unscaled product) folded
// in, so that the kernels below spend their issue slots on the tangents only (and, for S = float,
// never leave the FP32 pipe).  While relaxing, the species rows carry no transport and no anode term.
template <class S>
struct LinKT {
    S fD[6], fK[6], fKd[6], fKm[6];   // face: D0 and kappa_m (species row), K^d and K^m (Phi^L row)
    S vD[6], vK[6], vKd[6], vKm[6];   // volume: the same with the volume weight
    S fS, vS;                         // Phi^S: kappa_s at faces, 2 kappa_s in the volume
    S aLi, aL;                        // anode: k_Ano (Li+ row), F k_Ano (Phi^L row)
    S cl0, cl1, cr0, cr1;             // pen [[psi]] - {d_n psi} as weights of the four line values
    S rs[10];                         // row scales of the node part
    S c_pore, c_sep, phi;             // node diagonal of pore and separator voxels
    S wS[6], visc;                    // c_S weights and the viscosity coefficient (transport-factor tangents)
    int charged, sulfur;              // bit m: species m is charged / counts in c_S
};

template <class S>
static LinKT<S> make_link(const DevParams& p, int nl, int nf, int philf, int phisf, int relax, double dt,
                          double sc_dt) {
    LinKT<S> k;
    const double vol = 3.0 * p.h / 8.0, wf = 0.25 * p.h * p.h, h2 = 0.5 * SQ3 / p.h, pen = p.penalty / p.h;
    auto sc = [&](int f) { return sc_dt > 0.0 ? sc_dt * p.rscale[f] : 1.0; };
    const double sL = sc(philf), sS = sc(phisf);
    k.charged = 0;
    k.sulfur = 0;
    for (int m = 0; m < 6; ++m) {
        const bool on = m < nl;
        const double sm = on ? sc(m) : 0.0;
        const double D0 = on && !relax ? p.D0[m] : 0.0, km = on && !relax ? p.kappa_m[m] : 0.0;
        const double Kd = on ? p.Kd[m] : 0.0, Km = on ? p.Km[m] : 0.0;
        k.fD[m] = S(D0 * wf * sm); k.fK[m] = S(km * wf * sm); k.fKd[m] = S(Kd * wf * sL); k.fKm[m] = S(Km * wf * sL);
        k.vD[m] = S(D0 * vol * sm); k.vK[m] = S(km * vol * sm); k.vKd[m] = S(Kd * vol * sL); k.vKm[m] = S(Km * vol * sL);
        k.wS[m] = S(on ? p.wS[m] : 0.0);
        if (on && p.zc[m] != 0.0) k.charged |= 1 << m;
        if (on && p.wS[m] != 0.0) k.sulfur |= 1 << m;
    }
    k.fS = S(p.kappa_s * wf * sS);
    k.vS = S(2.0 * p.kappa_s * vol * sS);
    k.aLi = S(relax ? 0.0 : p.kAno * wf * sc(0));
    k.aL = S(p.F * p.kAno * wf * sL);
    // (ALPHA l1 + BETA l0 - ALPHA r0 - BETA r1) pen - h2 ((l1 - l0) + (r1 - r0))
    k.cl1 = S(ALPHA * pen - h2);
    k.cl0 = S(BETA * pen + h2);
    k.cr0 = S(-ALPHA * pen + h2);
    k.cr1 = S(-BETA * pen - h2);
    for (int f = 0; f < 10; ++f) k.rs[f] = S(f < nf ? sc(f) : 1.0);
    const NodeDiag nd = make_node_diag(p, dt, relax);
    k.c_pore = S(nd.c_pore);
    k.c_sep = S(nd.c_sep);
    k.phi = S(nd.phi);
    k.visc = S(p.visc);
    return k;
}

// tangents of the 32 transport factors of each voxel: dg = g (gam d eps_L - visc d c_S)
template <class Chem, class S>
__global__ void __launch_bounds__(128) k_lin_g(const DevParams p, const LinKT<S> K, const Geo g,
                                               const S* __restrict__ v, const S* __restrict__ gb,
                                               const S* __restrict__ gam, S* __restrict__ gbd) {
    int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= p.n_cell) return;
    constexpr int NL = Chem::NL, NS = Chem::NS;
    const int ph = g.phase[cell];
    const int s = g.cmap[cell];
    S dcs[8], del[8];
#pragma unroll
    for (int n = 0; n < 8; ++n) {
        S a = S(0);
#pragma unroll
        for (int m = 0; m < NL; ++m)
            if ((K.sulfur >> m) & 1) a += K.wS[m] * ld(v, p, m, n, cell);
        dcs[n] = a;
        del[n] = (NS == 2 && ph == 1) ? -(ld(v, p, NL, n, s) + ld(v, p, NL + 1, n, s)) : S(0);
        int64_t o = (int64_t)n * p.n_cell + cell;
        gbd[o] = gb[o] * (gam[o] * del[n] - K.visc * dcs[n]);
    }
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int side = -1; side <= 1; side += 2)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                int n0, n1;
                line_nodes(d, q, n0, n1);
                const S wn = side > 0 ? S(ALPHA) : S(BETA), wf = side > 0 ? S(BETA) : S(ALPHA);
                int64_t o = (int64_t)face_slot(d, side, q) * p.n_cell + cell;
                S dc = dcs[n1] * wn + dcs[n0] * wf;
                S de = del[n1] * wn + del[n0] * wf;
                gbd[o] = gb[o] * (gam[o] * de - K.visc * dc);
            }
}

// node part of the JVP: out = J_node v_node (writes; the line passes add).  Structure voxels and
// the others run in separate kernels so that no warp mixes the 10 x 10 product with the diagonal
// (on GB300 an FP64 instruction costs its issue slots whether or not all lanes take it).
// (a) one thread per (node, structure voxel), over the compact structure list
template <class Chem, class S>
__global__ void __launch_bounds__(128) k_lin_nodes_apply(const DevParams p, const LinKT<S> K, const Geo g,
                                                         const S* __restrict__ v, const S* __restrict__ jn,
                                                         S* __restrict__ out) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= (int64_t)p.n_struct * 8) return;
    constexpr int NF = Chem::NF;
    const int n = (int)(b / p.n_struct);
    const int sidx = (int)(b - (int64_t)n * p.n_struct);
    const int cell = g.sidx[sidx];
    S x[NF];
    int64_t idx[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        idx[f] = p.off[f] + (int64_t)n * p.flen[f] + (p.is_struct[f] ? sidx : cell);
        x[f] = v[idx[f]];
    }
    const S* J = jn + (int64_t)n * NF * NF * p.n_struct + sidx;
#pragma unroll
    for (int r = 0; r < NF; ++r) {
        S acc = S(0);
#pragma unroll
        for (int c = 0; c < NF; ++c) acc += J[(int64_t)(r * NF + c) * p.n_struct] * x[c];
        out[idx[r]] = acc * K.rs[r];
    }
}

// (b) one thread per (node, voxel): the storage diagonal of pore and separator voxels
template <class Chem, class S>
__global__ void __launch_bounds__(128) k_lin_nodes_diag(const DevParams p, const LinKT<S> K, const Geo g,
                                                        const S* __restrict__ v, S* __restrict__ out) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= (int64_t)p.n_cell * 8) return;
    constexpr int NL = Chem::NL, PHIL = Chem::PHIL;
    const int n = (int)(b / p.n_cell);
    const int cell = (int)(b - (int64_t)n * p.n_cell);
    const int ph = g.phase[cell];
    if (ph == 1) return;
    const S dc = ph == 2 ? K.c_sep : K.c_pore;
#pragma unroll
    for (int f = 0; f <= PHIL; ++f) {
        if (f >= NL && f != PHIL) continue;     // solid fields do not live here
        const int64_t idx = p.off[f] + (int64_t)n * p.flen[f] + cell;
        out[idx] = (f == PHIL ? K.phi : dc) * v[idx] * K.rs[f];
    }
}

// Face-once form of the line part: (1) one thread per +d face (voxel, line) computes the tangent of
// that face's fluxes for every transport equation once and stores them, already weighted and
// row-scaled; (2) one thread per (voxel, line) adds the volume terms and gathers its two faces.
// An interior face is evaluated once instead of once from each side.
// flux: [4 lines][NL + 2][n_cell] for the current direction.
template <class Chem, class S>
__global__ void __launch_bounds__(128) k_lin_face_flux(const DevParams p, const LinKT<S> K, const Geo g,
                                                       const S* __restrict__ v, const S* __restrict__ gbd,
                                                       const S* __restrict__ face, int d, S* __restrict__ flux) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= (int64_t)p.n_cell * 4) return;
    typedef LinShape<Chem> SH;
    constexpr int NL = Chem::NL;
    const S A_ = S(ALPHA), B_ = S(BETA);
    const int q = (int)(b / p.n_cell);
    const int cell = (int)(b - (int64_t)q * p.n_cell);
    int i, j, k;
    cell_ijk(p, cell, i, j, k);
    int n0, n1;
    line_nodes(d, q, n0, n1);
    const int coord = d == 0 ? i : d == 1 ? j : k;
    const int ext = d == 0 ? p.nx : d == 1 ? p.ny : p.nz;
    const int stride = d == 0 ? 1 : d == 1 ? p.nx : p.nx * p.ny;
    S* out = flux + (int64_t)q * (NL + 2) * p.n_cell + cell;
    auto put = [&](int e, S val) { out[(int64_t)e * p.n_cell] = val; };
    const S* Fd = face + (int64_t)((d * 4 + q) * SH::NFD) * p.n_cell + cell;
    auto F = [&](int kk) { return Fd[(int64_t)kk * p.n_cell]; };
    auto V = [&](int f, int n, int idx) { return v[p.off[f] + (int64_t)n * p.flen[f] + idx]; };
    if (coord + 1 >= ext) {
        // domain face: only the anode face (x = nx) carries a flux with a tangent
        S fLi = S(0), fL = S(0);
        if (d == 0) {
            S dcLi = A_ * V(0, n1, cell) + B_ * V(0, n0, cell);
            S dphL = A_ * V(Chem::PHIL, n1, cell) + B_ * V(Chem::PHIL, n0, cell);
            S drA = F(0) * dcLi + F(1) * dphL;
            fLi = drA * K.aLi;
            fL = drA * K.aL;
        }
        put(0, fLi);
        for (int e = 1; e < NL + 2; ++e) put(e, e == NL ? fL : S(0));
        return;
    }
    const int qc = cell + stride;
    const int64_t ol = (int64_t)face_slot(d, +1, q) * p.n_cell + cell, orr = (int64_t)face_slot(d, -1, q) * p.n_cell + qc;
    const S dgl = gbd[ol], dgr = gbd[orr];
    const S Hg = F(0), dHg = F(1) * dgl + F(2) * dgr;
    auto bracket = [&](S l0, S l1, S r0, S r1) { return K.cl1 * l1 + K.cl0 * l0 + K.cr0 * r0 + K.cr1 * r1; };
    const S BL = F(3 + NL);
    const S dBL = bracket(V(Chem::PHIL, n0, cell), V(Chem::PHIL, n1, cell), V(Chem::PHIL, n0, qc), V(Chem::PHIL, n1, qc));
    S fL = S(0);
#pragma unroll
    for (int m = 0; m < NL; ++m) {
        const S l0 = V(m, n0, cell), l1 = V(m, n1, cell), r0 = V(m, n0, qc), r1 = V(m, n1, qc);
        const S dterm = dHg * F(3 + m) + Hg * bracket(l0, l1, r0, r1);
        S f = dterm * K.fD[m];
        if ((K.charged >> m) & 1) {
            fL += dterm * K.fKd[m];
            const int base = 4 + NL + 5 * SH::ci(m);
            const S dcl = A_ * l1 + B_ * l0, dcr = A_ * r0 + B_ * r1;
            const S dHm = F(base + 1) * dgl + F(base + 2) * dcl + F(base + 3) * dgr + F(base + 4) * dcr;
            const S mterm = dHm * BL + F(base) * dBL;
            f += mterm * K.fK[m];
            fL += mterm * K.fKm[m];
        }
        put(m, f);
    }
    put(NL, fL);
    S fS = S(0);
    if (g.phase[cell] == 1 && g.phase[qc] == 1) {
        const int s = g.cmap[cell], sq = g.cmap[qc];
        fS = bracket(V(Chem::PHIS, n0, s), V(Chem::PHIS, n1, s), V(Chem::PHIS, n0, sq), V(Chem::PHIS, n1, sq)) * K.fS;
    }
    put(NL + 1, fS);
}

template <class Chem, class S>
__global__ void __launch_bounds__(128) k_lin_line_gather(const DevParams p, const LinKT<S> K, const Geo g,
                                                         const S* __restrict__ z, const S* __restrict__ v,
                                                         const S* __restrict__ gb, const S* __restrict__ gbd,
                                                         const S* __restrict__ flux, int d, S* __restrict__ out) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= (int64_t)p.n_cell * 4) return;
    constexpr int NL = Chem::NL;
    const S A_ = S(ALPHA), B_ = S(BETA);
    const int q = (int)(b / p.n_cell);
    const int cell = (int)(b - (int64_t)q * p.n_cell);
    int i, j, k;
    cell_ijk(p, cell, i, j, k);
    int n0, n1;
    line_nodes(d, q, n0, n1);
    const int coord = d == 0 ? i : d == 1 ? j : k;
    const int stride = d == 0 ? 1 : d == 1 ? p.nx : p.nx * p.ny;
    const bool hasL = coord > 0;
    const S* Fp = flux + (int64_t)q * (NL + 2) * p.n_cell + cell;                 // own +d face
    const S* Fm = flux + (int64_t)q * (NL + 2) * p.n_cell + (hasL ? cell - stride : cell);
    auto V = [&](int f, int n, int idx) { return v[p.off[f] + (int64_t)n * p.flen[f] + idx]; };
    auto Z = [&](int f, int n, int idx) { return z[p.off[f] + (int64_t)n * p.flen[f] + idx]; };
    // own face as left voxel adds +f (ALPHA to n1, BETA to n0); the -d face, where this voxel is the
    // right one, adds -f (ALPHA to n0, BETA to n1); fl is the volume flux along the line
    auto gather = [&](int e, int f, int idx, S fl) {
        const S fp = Fp[(int64_t)e * p.n_cell];
        const S fm = hasL ? Fm[(int64_t)e * p.n_cell] : S(0);
        const S o1 = fl + A_ * fp - B_ * fm;
        const S o0 = -fl + B_ * fp - A_ * fm;
        out[p.off[f] + (int64_t)n0 * p.flen[f] + idx] += o0;
        out[p.off[f] + (int64_t)n1 * p.flen[f] + idx] += o1;
    };
    const S gN0 = gb[(int64_t)n0 * p.n_cell + cell], gN1 = gb[(int64_t)n1 * p.n_cell + cell];
    const S dgN0 = gbd[(int64_t)n0 * p.n_cell + cell], dgN1 = gbd[(int64_t)n1 * p.n_cell + cell];
    const S dPhi = Z(Chem::PHIL, n1, cell) - Z(Chem::PHIL, n0, cell);
    const S ddPhi = V(Chem::PHIL, n1, cell) - V(Chem::PHIL, n0, cell);
    const S gsum = gN0 + gN1, dgsum = dgN0 + dgN1;
    S flL = S(0);
#pragma unroll
    for (int m = 0; m < NL; ++m) {
        const S C0 = Z(m, n0, cell), C1 = Z(m, n1, cell);
        const S dC0 = V(m, n0, cell), dC1 = V(m, n1, cell);
        const S A = dgsum * (C1 - C0) + gsum * (dC1 - dC0);     // tangent of g_sum dc
        S fl = A * K.vD[m];
        if ((K.charged >> m) & 1) {
            flL += A * K.vKd[m];
            const S msum = gN0 * C0 + gN1 * C1;
            const S dmsum = dgN0 * C0 + gN0 * dC0 + dgN1 * C1 + gN1 * dC1;
            const S B = dmsum * dPhi + msum * ddPhi;             // tangent of (g c)_sum dPhi
            fl += B * K.vK[m];
            flL += B * K.vKm[m];
        }
        gather(m, m, cell, fl);
    }
    gather(NL, Chem::PHIL, cell, flL);
    if (g.phase[cell] == 1) {
        const int sidx = g.cmap[cell];
        gather(NL + 1, Chem::PHIS, sidx, (V(Chem::PHIS, n1, sidx) - V(Chem::PHIS, n0, sidx)) * K.vS);
    }
}

// Per-node diagonal blocks of S J from the linearisation: column c of node n's block is the
// linearised operator applied to the unit tangent at (n, c), read at node n's rows.  That tangent
// touches the node terms (cached Jacobian), the transport factors of this voxel (node n and the
// face points of the three lines through n), the volume term of each of those lines and the two
// faces at the ends of each line, where node n enters through its trace (weight ALPHA or BETA)
// and the normal-derivative term (+-sqrt(3)/h).  Every column's tangent is a combination of five
// seeds, so one pass over the three lines accumulates the responses to them:
//   X, Y   the transport factors moving with a unit tangent of eps_L (X) or of c_S (Y): the
//          tangent of g at a point is g (gam d eps_L - visc d c_S);
//   Dd, DL a unit tangent of species m at node n itself: rows m and Phi^L;
//   Pp     a unit tangent of Phi^L at node n: the charged species rows and Phi^L;
//   dS     a unit tangent of Phi^S at node n: row Phi^S.
// Column c is then J[:, c] + (species c: wS_c Y + Dd/DL; solid: -X; Phi^L: Pp; Phi^S: dS).
// One thread per (node, voxel); FMAs only.
template <class Chem, class S>
__global__ void __launch_bounds__(128) k_lin_blk(const DevParams p, const Geo g, const S* __restrict__ z,
                                                 const S* __restrict__ gb, const S* __restrict__ gam,
                                                 const S* __restrict__ jn, const S* __restrict__ face, double dt,
                                                 int relax, const NodeDiag nd, double* __restrict__ blk) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= (int64_t)p.n_cell * 8) return;
    typedef LinShape<Chem> SH;
    constexpr int NL = Chem::NL, NS = Chem::NS, NF = Chem::NF, PHIL = Chem::PHIL, PHIS = Chem::PHIS;
    const int n = (int)(b / p.n_cell);
    const int cell = (int)(b - (int64_t)n * p.n_cell);
    int i, j, k;
    cell_ijk(p, cell, i, j, k);
    const int ph = g.phase[cell];
    const bool st = ph == 1;
    const int an[3] = {n & 1, (n >> 1) & 1, (n >> 2) & 1};
    const S vol = S(3.0 * p.h / 8.0), wf = S(0.25 * p.h * p.h), gq = S(SQ3 / p.h), pen = S(p.penalty / p.h);
    const S visc = S(p.visc);
    auto Z = [&](int f, int nn) { return z[p.off[f] + (int64_t)nn * p.flen[f] + cell]; };
    S X[NF], Y[NF], Pp[NF], Dd[NL], DL[NL], dS = S(0.0);
#pragma unroll
    for (int r = 0; r < NF; ++r) X[r] = Y[r] = Pp[r] = S(0.0);
#pragma unroll
    for (int m = 0; m < NL; ++m) Dd[m] = DL[m] = S(0.0);
    // tangent of g at node n per unit eps_L tangent (gxN) and per unit c_S tangent (gyN)
    const S gxN = gb[(int64_t)n * p.n_cell + cell] * gam[(int64_t)n * p.n_cell + cell];
    const S gyN = -gb[(int64_t)n * p.n_cell + cell] * visc;
#pragma unroll 1
    for (int d = 0; d < 3; ++d) {
        const int u = d == 0 ? an[1] : an[0];
        const int w = d == 2 ? an[1] : an[2];
        const int q = u + 2 * w;
        int n0, n1;
        line_nodes(d, q, n0, n1);
        const bool a1 = n == n1;
        const S sgn = a1 ? S(1.0) : -S(1.0);
        const int coord = d == 0 ? i : d == 1 ? j : k;
        const int ext = d == 0 ? p.nx : d == 1 ? p.ny : p.nz;
        const int stride = d == 0 ? 1 : d == 1 ? p.nx : p.nx * p.ny;
        // ---- volume term of the line
        {
            const S gN0 = gb[(int64_t)n0 * p.n_cell + cell], gN1 = gb[(int64_t)n1 * p.n_cell + cell];
            const S gown = a1 ? gN1 : gN0;
            const S dPhi = Z(PHIL, n1) - Z(PHIL, n0);
            const S gsum = gN0 + gN1;
            const S sv = sgn * vol;
            S fLg = S(0.0), fLp = S(0.0);
#pragma unroll
            for (int m = 0; m < NL; ++m) {
                const S C0 = Z(m, n0), C1 = Z(m, n1);
                const S dc = C1 - C0, Cown = a1 ? C1 : C0;
                // transport-factor seed: d gsum = d g_n, d msum = d g_n C_n (per unit d g_n)
                S fg = relax ? S(0.0) : dc * S(p.D0[m]);
                // own-species seed: d dc = sgn, d msum = g_n
                S fd = relax ? S(0.0) : gsum * sgn * S(p.D0[m]);
                S fLd = S(0.0);
                if (p.zc[m] != S(0.0)) {
                    const S msum = gN0 * C0 + gN1 * C1;
                    if (!relax) {
                        fg += Cown * dPhi * S(p.kappa_m[m]);
                        fd += gown * dPhi * S(p.kappa_m[m]);
                        Pp[m] += msum * sgn * S(p.kappa_m[m]) * sv;     // Phi^L seed: d dPhi = sgn
                    }
                    fLg += dc * S(p.Kd[m]) + Cown * dPhi * S(p.Km[m]);
                    fLd = gsum * sgn * S(p.Kd[m]) + gown * dPhi * S(p.Km[m]);
                    fLp += msum * sgn * S(p.Km[m]);
                }
                X[m] += fg * gxN * sv;
                Y[m] += fg * gyN * sv;
                Dd[m] += fd * sv;
                DL[m] += fLd * sv;
            }
            X[PHIL] += fLg * gxN * sv;
            Y[PHIL] += fLg * gyN * sv;
            Pp[PHIL] += fLp * sv;
            if (st) dS += S(2.0) * S(p.kappa_s) * vol;
        }
        // ---- the two faces of the line: own voxel left (+d face) or right (-d face)
#pragma unroll 1
        for (int side = 1; side >= -1; side -= 2) {
            const bool left = side > 0;
            const S tw = left ? (a1 ? S(ALPHA) : S(BETA)) : (a1 ? S(BETA) : S(ALPHA));   // own trace weight
            const S dBown = left ? tw * pen - S(0.5) * gq * sgn : -tw * pen - S(0.5) * gq * sgn;
            const S wrow = left ? wf * tw : -wf * tw;
            const bool inside = left ? coord + 1 < ext : coord > 0;
            if (!inside) {
                if (left && d == 0) {   // anode face: r_Ano(c_Li, Phi^L) at the face point
                    const S* Fo = face + (int64_t)((d * 4 + q) * SH::NFD) * p.n_cell + cell;
                    const S drc = Fo[0] * tw, drp = Fo[(int64_t)p.n_cell] * tw;
                    if (!relax) {
                        Dd[0] += drc * S(p.kAno) * wrow;
                        Pp[0] += drp * S(p.kAno) * wrow;
                    }
                    DL[0] += drc * S(p.F) * S(p.kAno) * wrow;
                    Pp[PHIL] += drp * S(p.F) * S(p.kAno) * wrow;
                }
                continue;
            }
            const int fc = left ? cell : cell - stride;        // voxel owning the face data
            const int oc = left ? cell + stride : cell - stride;   // the other voxel
            const S* Fd = face + (int64_t)((d * 4 + q) * SH::NFD) * p.n_cell + fc;
            auto F = [&](int kk) { return Fd[(int64_t)kk * p.n_cell]; };
            const int64_t so = (int64_t)face_slot(d, side, q) * p.n_cell + cell;
            const S gxo = gb[so] * gam[so] * tw, gyo = -gb[so] * visc * tw;   // own g tangent per seed
            const S dHg1 = left ? F(1) : F(2);                   // d Hg per unit own g tangent
            const S Hg = F(0), BL = F(3 + NL);
            S fLg = S(0.0), fLp = S(0.0);
#pragma unroll
            for (int m = 0; m < NL; ++m) {
                const S tg = dHg1 * F(3 + m);                    // transport-factor seed
                const S td = Hg * dBown;                         // own-species seed (d B = dBown)
                S fg = relax ? S(0.0) : tg * S(p.D0[m]);
                S fd = relax ? S(0.0) : td * S(p.D0[m]);
                if (p.zc[m] != S(0.0)) {
                    const int base = 4 + NL + 5 * SH::ci(m);
                    const S mg = (left ? F(base + 1) : F(base + 3)) * BL;
                    const S md = (left ? F(base + 2) : F(base + 4)) * tw * BL;
                    const S mp = F(base) * dBown;                // Phi^L seed (d BL = dBown)
                    if (!relax) {
                        fg += mg * S(p.kappa_m[m]);
                        fd += md * S(p.kappa_m[m]);
                        Pp[m] += mp * S(p.kappa_m[m]) * wrow;
                    }
                    fLg += tg * S(p.Kd[m]) + mg * S(p.Km[m]);
                    DL[m] += (td * S(p.Kd[m]) + md * S(p.Km[m])) * wrow;
                    fLp += mp * S(p.Km[m]);
                }
                X[m] += fg * gxo * wrow;
                Y[m] += fg * gyo * wrow;
                Dd[m] += fd * wrow;
            }
            X[PHIL] += fLg * gxo * wrow;
            Y[PHIL] += fLg * gyo * wrow;
            Pp[PHIL] += fLp * wrow;
            if (st && g.phase[oc] == 1) dS += dBown * S(p.kappa_s) * wrow;
        }
    }
    const S* J = st ? jn + (int64_t)n * NF * NF * p.n_struct + g.cmap[cell] : nullptr;
    const S ddc = S(ph == 2 ? nd.c_sep : nd.c_pore), ddphi = S(nd.phi);
    double* B = blk + b * NF * NF;
#pragma unroll 1
    for (int c = 0; c < NF; ++c) {
        if (p.is_struct[c] && !st) {
            for (int r = 0; r < NF; ++r) B[r * NF + c] = r == c ? 1.0 : 0.0;
            continue;
        }
        S col[NF];
        if (st) {
#pragma unroll
            for (int r = 0; r < NF; ++r) col[r] = S(J[(int64_t)(r * NF + c) * p.n_struct]);
        } else {
#pragma unroll
            for (int r = 0; r < NF; ++r) col[r] = r != c ? S(0.0) : (r < NL ? ddc : (r == PHIL ? ddphi : S(0.0)));
        }
        if (c < NL) {
            const S dcs = S(p.wS[c]);                            // tangent of c_S
#pragma unroll
            for (int r = 0; r < NF; ++r) col[r] += dcs * Y[r];
#pragma unroll
            for (int m = 0; m < NL; ++m)
                if (m == c) { col[m] += Dd[m]; col[PHIL] += DL[m]; }
        } else if (c == PHIL) {
#pragma unroll
            for (int r = 0; r < NF; ++r) col[r] += Pp[r];
        } else if (c == PHIS) {
            col[PHIS] += dS;
        } else if (NS == 2 && st) {                              // a solid fraction: d eps_L = -1
#pragma unroll
            for (int r = 0; r < NF; ++r) col[r] -= X[r];
        }
#pragma unroll
        for (int r = 0; r < NF; ++r) {
            double o = double(col[r]) * dt * p.rscale[r];
            if (p.is_struct[r] && !st) o = r == c ? 1.0 : 0.0;
            B[r * NF + c] = o;
        }
    }
}

int64_t dg1_lin_sizes(const DevParams& p, int64_t* jn, int64_t* gam, int64_t* face) {
    const int nf = p.nf;
    const int nl = p.nl;
    const int nfd = 3 + nl + 1 + 5 * (nl - 1);
    *jn = (int64_t)8 * nf * nf * (p.n_struct > 0 ? p.n_struct : 1);
    *gam = (int64_t)NG * p.n_cell;
    *face = (int64_t)12 * nfd * p.n_cell;
    return (*jn + *gam + *face) * 8;
}

int64_t dg1_lin_flux_len(const DevParams& p) { return (int64_t)4 * (p.nl + 2) * p.n_cell;
}

template <class Chem, class S>
static cudaError_t linearize_impl(const LaunchCtx& L, const DevParams& p, const Geo& g, const S* z, double t,
                                  double dt, int relax, S* jn, S* gam, S* face, S* gb) {
    k_dg1_g<Chem, S, false><<<nblocks(p.n_cell, 128), 128, 0, L.st>>>(p, g, z, z, gb, gb);
    k_lin_gam<Chem, S><<<nblocks(p.n_cell, 128), 128, 0, L.st>>>(p, g, z, gam);
    if (p.n_struct > 0)
        k_lin_nodes_build<Chem, S><<<nblocks((int64_t)p.n_struct * 8, 64), 64, 0, L.st>>>(p, g, z, t, dt, relax, jn);
    for (int d = 0; d < 3; ++d)
        k_lin_faces_build<Chem, S><<<nblocks((int64_t)p.n_cell * 4, 128), 128, 0, L.st>>>(p, g, z, gb, d, face);
    *L.counter += 6;
    return cudaGetLastError();
}

// Linearise at z: in FP64, or (lin.f32, the mixed-precision path, whose products and blocks are FP32)
// in FP32 from an FP32 copy of z.
cudaError_t dg1_linearize(const LaunchCtx& L, const DevParams& p, const Geo& g, const double* z, double t, double dt,
                          int relax, const DG1Lin& lin) {
    if (lin.f32) {
        cudaError_t e = to_f32(L, lin.z32, z, lin.ndof);
        if (e != cudaSuccess) return e;
        return p.nf == 10 ? linearize_impl<ChemTO, float>(L, p, g, lin.z32, t, dt, relax, lin.jn32, lin.gam32, lin.face32,
                                                          lin.gb32)
                          : linearize_impl<ChemR3, float>(L, p, g, lin.z32, t, dt, relax, lin.jn32, lin.gam32, lin.face32,
                                                          lin.gb32);
    }
    return p.nf == 10 ? linearize_impl<ChemTO, double>(L, p, g, z, t, dt, relax, lin.jn, lin.gam, lin.face, lin.gb)
                      : linearize_impl<ChemR3, double>(L, p, g, z, t, dt, relax, lin.jn, lin.gam, lin.face, lin.gb);
}

template <class Chem, class S>
static cudaError_t lin_apply_impl(const LaunchCtx& L, const DevParams& p, const Geo& g, const S* z, const S* v,
                                  double dt, int relax, double sc_dt, S* out, const S* jn, const S* gam, const S* face,
                                  const S* gb, S* gbd, S* flux) {
    const LinKT<S> K = make_link<S>(p, Chem::NL, Chem::NF, Chem::PHIL, Chem::PHIS, relax, dt, sc_dt);
    k_lin_g<Chem, S><<<nblocks(p.n_cell, 128), 128, 0, L.st>>>(p, K, g, v, gb, gam, gbd);
    if (p.n_struct > 0)
        k_lin_nodes_apply<Chem, S><<<nblocks((int64_t)p.n_struct * 8, 128), 128, 0, L.st>>>(p, K, g, v, jn, out);
    k_lin_nodes_diag<Chem, S><<<nblocks((int64_t)p.n_cell * 8, 128), 128, 0, L.st>>>(p, K, g, v, out);
    for (int d = 0; d < 3; ++d) {
        k_lin_face_flux<Chem, S><<<nblocks((int64_t)p.n_cell * 4, 128), 128, 0, L.st>>>(p, K, g, v, gbd, face, d, flux);
        k_lin_line_gather<Chem, S><<<nblocks((int64_t)p.n_cell * 4, 128), 128, 0, L.st>>>(p, K, g, z, v, gb, gbd, flux, d,
                                                                                           out);
    }
    *L.counter += 9;
    return cudaGetLastError();
}

template <>
cudaError_t dg1_lin_apply<double>(const LaunchCtx& L, const DevParams& p, const Geo& g, const double* z, const double* v,
                                  double t, double dt, int relax, double sc_dt, double* out, const DG1Lin& lin) {
    if (lin.f32) return cudaErrorInvalidValue;
    return p.nf == 10 ? lin_apply_impl<ChemTO, double>(L, p, g, z, v, dt, relax, sc_dt, out, lin.jn, lin.gam, lin.face,
                                                       lin.gb, lin.gbd, lin.flux)
                      : lin_apply_impl<ChemR3, double>(L, p, g, z, v, dt, relax, sc_dt, out, lin.jn, lin.gam, lin.face,
                                                       lin.gb, lin.gbd, lin.flux);
}

template <>
cudaError_t dg1_lin_apply<float>(const LaunchCtx& L, const DevParams& p, const Geo& g, const float* z, const float* v,
                                 double t, double dt, int relax, double sc_dt, float* out, const DG1Lin& lin) {
    if (!lin.f32) return cudaErrorInvalidValue;
    return p.nf == 10 ? lin_apply_impl<ChemTO, float>(L, p, g, z, v, dt, relax, sc_dt, out, lin.jn32, lin.gam32,
                                                      lin.face32, lin.gb32, lin.gbd32, lin.flux32)
                      : lin_apply_impl<ChemR3, float>(L, p, g, z, v, dt, relax, sc_dt, out, lin.jn32, lin.gam32,
                                                      lin.face32, lin.gb32, lin.gbd32, lin.flux32);
}

cudaError_t dg1_lin_blocks(const LaunchCtx& L, const DevParams& p, const Geo& g, const double* z, double dt, int relax,
                           const DG1Lin& lin, double* blk) {
    const int nb = nblocks((int64_t)p.n_cell * 8, 128);
    const NodeDiag nd = make_node_diag(p, dt, relax);
    if (lin.f32) {   // FP32 arithmetic on the FP32 linearisation (the blocks only precondition an FP32 loop)
        if (p.nf == 10)
            k_lin_blk<ChemTO, float><<<nb, 128, 0, L.st>>>(p, g, lin.z32, lin.gb32, lin.gam32, lin.jn32, lin.face32, dt,
                                                           relax, nd, blk);
        else
            k_lin_blk<ChemR3, float><<<nb, 128, 0, L.st>>>(p, g, lin.z32, lin.gb32, lin.gam32, lin.jn32, lin.face32, dt,
                                                           relax, nd, blk);
    } else {
        if (p.nf == 10)
            k_lin_blk<ChemTO, double><<<nb, 128, 0, L.st>>>(p, g, z, lin.gb, lin.gam, lin.jn, lin.face, dt, relax, nd, blk);
        else
            k_lin_blk<ChemR3, double><<<nb, 128, 0, L.st>>>(p, g, z, lin.gb, lin.gam, lin.jn, lin.face, dt, relax, nd, blk);
    }
    *L.counter += 1;
    return cudaGetLastError();
}

// ------------------------------------------------------------------ slope limiter
// Vertex-based slope limiter (App. B, after Kuzmin 2010) on the conserved densities q = eps_L c of
// the liquid species: per voxel and species the deviation of q from its voxel mean is scaled by the
// largest factor in [0, 1] that keeps the Q1 field at each of the 8 voxel corners within the range of
// the means of the voxels sharing that corner.  Voxel means (hence every species) are unchanged.
template <class Chem>
__device__ __forceinline__ void node_eps_l(const DevParams& p, const Geo& g, const double* z, int cell, double* eL) {
    const int ph = g.phase[cell];
    const int s = g.cmap[cell];
#pragma unroll
    for (int n = 0; n < 8; ++n) {
        double es[2] = {0.0, 0.0};
        if (Chem::NS == 2 && ph == 1) {
            es[0] = ld(z, p, Chem::NL, n, s);
            es[1] = ld(z, p, Chem::NL + 1, n, s);
        }
        eL[n] = liquid_fraction<Chem, double>(p, ph, es);
    }
}

template <class Chem>
__global__ void __launch_bounds__(128) k_lim_means(const DevParams p, const Geo g, const double* __restrict__ z,
                                                   double* __restrict__ mean) {
    int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= p.n_cell) return;
    double eL[8];
    node_eps_l<Chem>(p, g, z, cell, eL);
#pragma unroll 1
    for (int m = 0; m < Chem::NL; ++m) {
        double acc = 0.0;
#pragma unroll
        for (int n = 0; n < 8; ++n) acc += eL[n] * ld(z, p, m, n, cell);
        mean[(int64_t)m * p.n_cell + cell] = acc / 8.0;
    }
}

template <class Chem>
__global__ void __launch_bounds__(128) k_lim_apply(const DevParams p, const Geo g, const double* __restrict__ mean,
                                                   double* __restrict__ z) {
    int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= p.n_cell) return;
    int i, j, k;
    cell_ijk(p, cell, i, j, k);
    double eL[8];
    node_eps_l<Chem>(p, g, z, cell, eL);
    const double W[2][2] = {{ALPHA, BETA}, {BETA, ALPHA}};   // W[corner side][node side]
#pragma unroll 1
    for (int m = 0; m < Chem::NL; ++m) {
        const double* M = mean + (int64_t)m * p.n_cell;
        const double qbar = M[cell];
        double q[8];
#pragma unroll
        for (int n = 0; n < 8; ++n) q[n] = eL[n] * ld(z, p, m, n, cell);
        double alpha = 1.0;
#pragma unroll 1
        for (int c = 0; c < 8; ++c) {
            const int cx = c & 1, cy = (c >> 1) & 1, cz = c >> 2;
            double uc = 0.0;
#pragma unroll
            for (int n = 0; n < 8; ++n) uc += W[cx][n & 1] * W[cy][(n >> 1) & 1] * W[cz][n >> 2] * q[n];
            double vmax = -INFINITY, vmin = INFINITY;
            for (int kk = k + cz - 1; kk <= k + cz; ++kk) {
                if (kk < 0 || kk >= p.nz) continue;
                for (int jj = j + cy - 1; jj <= j + cy; ++jj) {
                    if (jj < 0 || jj >= p.ny) continue;
                    for (int ii = i + cx - 1; ii <= i + cx; ++ii) {
                        if (ii < 0 || ii >= p.nx) continue;
                        const double v = M[ii + (int64_t)p.nx * (jj + (int64_t)p.ny * kk)];
                        vmax = fmax(vmax, v);
                        vmin = fmin(vmin, v);
                    }
                }
            }
            const double d = uc - qbar;
            if (d > 0.0) alpha = fmin(alpha, fmin(1.0, (vmax - qbar) / d));
            else if (d < 0.0) alpha = fmin(alpha, fmin(1.0, (vmin - qbar) / d));
        }
        if (alpha < 1.0) {
#pragma unroll
            for (int n = 0; n < 8; ++n)
                z[p.off[m] + (int64_t)n * p.flen[m] + cell] = (qbar + alpha * (q[n] - qbar)) / eL[n];
        }
    }
}

cudaError_t dg1_limit(const LaunchCtx& L, const DevParams& p, const Geo& g, double* z, double* scratch) {
    const int nb = nblocks(p.n_cell, 128);
    if (p.nf == 10) {
        k_lim_means<ChemTO><<<nb, 128, 0, L.st>>>(p, g, z, scratch);
        k_lim_apply<ChemTO><<<nb, 128, 0, L.st>>>(p, g, scratch, z);
    } else {
        k_lim_means<ChemR3><<<nb, 128, 0, L.st>>>(p, g, z, scratch);
        k_lim_apply<ChemR3><<<nb, 128, 0, L.st>>>(p, g, scratch, z);
    }
    *L.counter += 2;
    return cudaGetLastError();
}

// ------------------------------------------------------------------ launchers

// ------------------------------------------------------------------ residual, each face once
// (1) one thread per +d face (voxel, nodal line): the weighted fluxes of every transport equation
// through that face (and the anode exchange on the x = nx face); (2) one thread per (voxel, line):
// the volume terms of the line, plus its two faces, plus the collector current on the x = 0 face.
// flux: [4 lines][NL + 2][n_cell] for the current direction.
template <class Chem>
__global__ void __launch_bounds__(128) k_res_face(const DevParams p, const Geo g, const double* __restrict__ z,
                                                  const double* __restrict__ gb, int d, int relax,
                                                  double* __restrict__ flux) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= (int64_t)p.n_cell * 4) return;
    constexpr int NL = Chem::NL;
    const int q = (int)(b / p.n_cell);
    const int cell = (int)(b - (int64_t)q * p.n_cell);
    int i, j, k;
    cell_ijk(p, cell, i, j, k);
    int n0, n1;
    line_nodes(d, q, n0, n1);
    const double wf = 0.25 * p.h * p.h, gq = SQ3 / p.h, pen = p.penalty / p.h;
    const double al = ALPHA, be = BETA;
    const int coord = d == 0 ? i : d == 1 ? j : k;
    const int ext = d == 0 ? p.nx : d == 1 ? p.ny : p.nz;
    const int stride = d == 0 ? 1 : d == 1 ? p.nx : p.nx * p.ny;
    double* out = flux + (int64_t)q * (NL + 2) * p.n_cell + cell;
    auto put = [&](int e, double val) { out[(int64_t)e * p.n_cell] = val; };
    auto Z = [&](int f, int n, int idx) { return z[p.off[f] + (int64_t)n * p.flen[f] + idx]; };
    if (coord + 1 >= ext) {
        double fLi = 0.0, fL = 0.0;
        if (d == 0) {   // anode exchange at the face points of the x = nx face
            const double cLi = Z(0, n1, cell) * al + Z(0, n0, cell) * be;
            const double phL = Z(Chem::PHIL, n1, cell) * al + Z(Chem::PHIL, n0, cell) * be;
            const double rA = anode_rate<double>(p, cLi, phL);
            if (!relax) fLi = rA * (wf * p.kAno);
            fL = rA * (wf * (p.F * p.kAno));
        }
        put(0, fLi);
        for (int e = 1; e < NL + 2; ++e) put(e, e == NL ? fL : 0.0);
        return;
    }
    const int qc = cell + stride;
    const double gl = gb[(int64_t)face_slot(d, +1, q) * p.n_cell + cell];
    const double gr = gb[(int64_t)face_slot(d, -1, q) * p.n_cell + qc];
    const double Hg = harm(gl, gr);
    const double PL0 = Z(Chem::PHIL, n0, cell), PL1 = Z(Chem::PHIL, n1, cell);
    const double PQ0 = Z(Chem::PHIL, n0, qc), PQ1 = Z(Chem::PHIL, n1, qc);
    const double jL = (PL1 * al + PL0 * be) - (PQ0 * al + PQ1 * be);
    const double mL = ((PL1 - PL0) + (PQ1 - PQ0)) * (gq * 0.5);
    double fL = 0.0;
#pragma unroll 1
    for (int m = 0; m < NL; ++m) {
        const double C0 = Z(m, n0, cell), C1 = Z(m, n1, cell), Q0 = Z(m, n0, qc), Q1 = Z(m, n1, qc);
        const double tP = C1 * al + C0 * be, tN = Q0 * al + Q1 * be;
        const double mc = ((C1 - C0) + (Q1 - Q0)) * (gq * 0.5);
        const double dterm = ((tP - tN) * pen - mc) * Hg;
        double f = relax ? 0.0 : dterm * p.D0[m];
        if (p.zc[m] != 0.0) {
            const double Hm = harm(gl * tP, gr * tN);
            const double mterm = (jL * pen - mL) * Hm;
            if (!relax) f += mterm * p.kappa_m[m];
            fL += dterm * p.Kd[m] + mterm * p.Km[m];
        }
        put(m, f * wf);
    }
    put(NL, fL * wf);
    double fS = 0.0;
    if (g.phase[cell] == 1 && g.phase[qc] == 1) {
        const int s = g.cmap[cell], sq = g.cmap[qc];
        const double S0 = Z(Chem::PHIS, n0, s), S1 = Z(Chem::PHIS, n1, s);
        const double Q0 = Z(Chem::PHIS, n0, sq), Q1 = Z(Chem::PHIS, n1, sq);
        const double jS = (S1 * al + S0 * be) - (Q0 * al + Q1 * be);
        const double mS = ((S1 - S0) + (Q1 - Q0)) * (gq * 0.5);
        fS = (jS * pen - mS) * p.kappa_s * wf;
    }
    put(NL + 1, fS);
}

template <class Chem>
__global__ void __launch_bounds__(128) k_res_gather(const DevParams p, const Geo g, const double* __restrict__ z,
                                                    const double* __restrict__ gb, const double* __restrict__ flux, int d,
                                                    double t, int relax, double* __restrict__ r) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= (int64_t)p.n_cell * 4) return;
    constexpr int NL = Chem::NL;
    const int q = (int)(b / p.n_cell);
    const int cell = (int)(b - (int64_t)q * p.n_cell);
    int i, j, k;
    cell_ijk(p, cell, i, j, k);
    int n0, n1;
    line_nodes(d, q, n0, n1);
    const double vol = 3.0 * p.h / 8.0;
    const int coord = d == 0 ? i : d == 1 ? j : k;
    const int stride = d == 0 ? 1 : d == 1 ? p.nx : p.nx * p.ny;
    const bool hasL = coord > 0;
    const double* Fp = flux + (int64_t)q * (NL + 2) * p.n_cell + cell;
    const double* Fm = flux + (int64_t)q * (NL + 2) * p.n_cell + (hasL ? cell - stride : cell);
    auto Z = [&](int f, int n, int idx) { return z[p.off[f] + (int64_t)n * p.flen[f] + idx]; };
    auto gather = [&](int e, int f, int idx, double a0, double a1) {
        const double fp = Fp[(int64_t)e * p.n_cell];
        const double fm = hasL ? Fm[(int64_t)e * p.n_cell] : 0.0;
        a1 += fp * ALPHA - fm * BETA;
        a0 += fp * BETA - fm * ALPHA;
        r[p.off[f] + (int64_t)n0 * p.flen[f] + idx] += a0;
        r[p.off[f] + (int64_t)n1 * p.flen[f] + idx] += a1;
    };
    const double gN0 = gb[(int64_t)n0 * p.n_cell + cell], gN1 = gb[(int64_t)n1 * p.n_cell + cell];
    const double gsum = gN0 + gN1;
    const double dPhi = Z(Chem::PHIL, n1, cell) - Z(Chem::PHIL, n0, cell);
    double accL = 0.0;
#pragma unroll 1
    for (int m = 0; m < NL; ++m) {
        const double C0 = Z(m, n0, cell), C1 = Z(m, n1, cell);
        const double dc = C1 - C0;
        double fl = relax ? 0.0 : gsum * dc * p.D0[m];
        if (p.zc[m] != 0.0) {
            const double msum = gN0 * C0 + gN1 * C1;
            if (!relax) fl += msum * dPhi * p.kappa_m[m];
            accL += (gsum * dc * p.Kd[m] + msum * dPhi * p.Km[m]) * vol;
        }
        fl = fl * vol;
        gather(m, m, cell, -fl, fl);
    }
    gather(NL, Chem::PHIL, cell, -accL, accL);
    if (g.phase[cell] == 1) {
        const int sidx = g.cmap[cell];
        const double fs = (Z(Chem::PHIS, n1, sidx) - Z(Chem::PHIS, n0, sidx)) * (2.0 * p.kappa_s * vol);
        double a0 = -fs, a1 = fs;
        if (d == 0 && i == 0) {   // collector current on the x = 0 face (ramped while relaxing)
            const double fj = 0.25 * p.h * p.h * p.j_cc * (relax ? smooth_step(t) : 1.0);
            a0 += fj * ALPHA;
            a1 += fj * BETA;
        }
        gather(NL + 1, Chem::PHIS, sidx, a0, a1);
    }
}

int64_t dg1_face_buffer_len(const DevParams& p) { return (int64_t)NG * p.n_cell; }

template <class Chem>
static cudaError_t residual_impl(const LaunchCtx& L, const DevParams& p, const Geo& g, const double* z, const double* zn,
                                 double t, double dt, int relax, double* r, double* gb, double* flux) {
    k_dg1_g<Chem, double, false><<<nblocks(p.n_cell, 128), 128, 0, L.st>>>(p, g, z, z, gb, gb);
    k_dg1_nodes<Chem, double, 0><<<nblocks((int64_t)p.n_cell * 8, 128), 128, 0, L.st>>>(p, g, z, z, zn, t, dt, relax, 0.0, r);
    for (int d = 0; d < 3; ++d) {
        k_res_face<Chem><<<nblocks((int64_t)p.n_cell * 4, 128), 128, 0, L.st>>>(p, g, z, gb, d, relax, flux);
        k_res_gather<Chem><<<nblocks((int64_t)p.n_cell * 4, 128), 128, 0, L.st>>>(p, g, z, gb, flux, d, t, relax, r);
    }
    *L.counter += 8;
    return cudaGetLastError();
}

// flux: scratch of at least 4 (NL + 2) n_cell doubles
cudaError_t dg1_residual(const LaunchCtx& L, const DevParams& p, const Geo& g, const double* z, const double* zn,
                         double t, double dt, int relax, double* r, double* gb, double* flux) {
    return p.nf == 10 ? residual_impl<ChemTO>(L, p, g, z, zn, t, dt, relax, r, gb, flux)
                      : residual_impl<ChemR3>(L, p, g, z, zn, t, dt, relax, r, gb, flux);
}

template <class Chem, class S>
static cudaError_t jvp_impl(const LaunchCtx& L, const DevParams& p, const Geo& g, const S* z, const S* v, double t,
                            double dt, int relax, double sc_dt, S* out, S* gb, S* gbd) {
    k_dg1_g<Chem, S, true><<<nblocks(p.n_cell, 128), 128, 0, L.st>>>(p, g, z, v, gb, gbd);
    k_dg1_nodes<Chem, S, 1><<<nblocks((int64_t)p.n_cell * 8, 128), 128, 0, L.st>>>(p, g, z, v, nullptr, t, dt, relax, sc_dt, out);
    for (int d = 0; d < 3; ++d)
        k_dg1_lines<Chem, S, 1><<<nblocks((int64_t)p.n_cell * 4, 128), 128, 0, L.st>>>(p, g, z, v, gb, gbd, d, t, dt, relax, sc_dt, out);
    *L.counter += 5;
    return cudaGetLastError();
}

template <class S>
cudaError_t dg1_jvp(const LaunchCtx& L, const DevParams& p, const Geo& g, const S* z, const S* v, double t, double dt,
                    int relax, double sc_dt, S* out, S* gb, S* gbd) {
    return p.nf == 10 ? jvp_impl<ChemTO, S>(L, p, g, z, v, t, dt, relax, sc_dt, out, gb, gbd)
                      : jvp_impl<ChemR3, S>(L, p, g, z, v, t, dt, relax, sc_dt, out, gb, gbd);
}
template cudaError_t dg1_jvp<double>(const LaunchCtx&, const DevParams&, const Geo&, const double*, const double*, double,
                                     double, int, double, double*, double*, double*);
template cudaError_t dg1_jvp<float>(const LaunchCtx&, const DevParams&, const Geo&, const float*, const float*, double,
                                    double, int, double, float*, float*, float*);


cudaError_t dg1_gfactor(const LaunchCtx& L, const DevParams& p, const Geo& g, const double* z, double* gb) {
    if (p.nf == 10) k_dg1_g<ChemTO, double, false><<<nblocks(p.n_cell, 128), 128, 0, L.st>>>(p, g, z, z, gb, gb);
    else k_dg1_g<ChemR3, double, false><<<nblocks(p.n_cell, 128), 128, 0, L.st>>>(p, g, z, z, gb, gb);
    *L.counter += 1;
    return cudaGetLastError();
}

}  // namespace dgls
