// DG0 (p = 0) residual, Jacobian-vector product and diagonal Jacobian blocks of the Li-S model.
//
// Eq. 48 applied component-wise to Tab. 4: every interior face contributes
// A {K}_H (psi_P - psi_Q)/h per (coefficient x gradient) term.  All coefficients of the liquid
// phase are a constant times g = eps_L^{3/2} eta(0)/eta(c_S) or times g c_i, and the harmonic
// mean is homogeneous of degree one, so each face needs only H(g_P, g_Q) and, per charged
// species, H(g_P c_iP, g_Q c_iQ): 1 + (charged species) divisions per face instead of one per
// term.
//
// Launch shape: one thread per voxel (x fastest, so warps read contiguous x-runs of every
// field); a first pass stores g (and its tangent) per voxel so that neighbours do not
// recompute the viscosity exponential; each thread then evaluates its own reactions once and
// its six faces.
#include <algorithm>

#include "internal.h"

namespace dgls {

template <class Chem, class T>
struct CellVals {
    T c[Chem::NL];
    T es[2];
    T phiL, phiS;
    T g;
    int ph;
    int sidx;
};

__device__ __forceinline__ void cell_ijk(const DevParams& p, int cell, int& i, int& j, int& k) {
    i = cell % p.nx;
    int r = cell / p.nx;
    j = r % p.ny;
    k = r / p.ny;
}

// Residual rows of voxel P (volume-integrated, unscaled); old[] holds z^n of P's fields
// (zeros when only tangents are wanted).
template <class Chem, class T, class GetQ>
__device__ __forceinline__ void dg0_cell(const DevParams& p, int i, int j, int k, const CellVals<Chem, T>& P,
                                         GetQ getQ, const double* old, double tH, double jscale, double dt,
                                         int relax, T* R) {
    typedef typename Base<T>::type Sc;
    constexpr int NL = Chem::NL, NS = Chem::NS, PHIL = Chem::PHIL, PHIS = Chem::PHIS;
    const bool st = (P.ph == 1);
    const Sc h = Sc(p.h);
    const Sc Vdt = Sc(p.V / dt);
#pragma unroll
    for (int f = 0; f < Chem::NF; ++f) R[f] = Make<T>::c(0.0);

    // ---- storage: V (eps_L c - eps_L^n c^n)/dt, V rho/M (eps - eps^n)/dt, relaxation d_t Phi
    T epsL = liquid_fraction<Chem, T>(p, P.ph, P.es);
    double esn[2] = {0.0, 0.0};
    if (NS == 2) { esn[0] = old[NL]; esn[1] = old[NL + 1]; }
    double epsLn = val(liquid_fraction<Chem, double>(p, P.ph, esn));
#pragma unroll
    for (int m = 0; m < NL; ++m) {
        if (relax) R[m] = (P.c[m] - Make<T>::c(old[m])) * Vdt;
        else R[m] = (epsL * P.c[m] - Make<T>::c(epsLn * old[m])) * Vdt;
    }
    if (st) {
#pragma unroll
        for (int s = 0; s < NS; ++s) R[NL + s] = (P.es[s] - Make<T>::c(old[NL + s])) * Sc(p.V * p.rhoM[s] / dt);
    }
    if (relax) {
        R[PHIL] = (P.phiL - Make<T>::c(old[PHIL])) * Vdt;
        if (st) R[PHIS] = (P.phiS - Make<T>::c(old[PHIS])) * Vdt;
    }

    // ---- faces
#pragma unroll 1
    for (int d = 0; d < 6; ++d) {
        int qi = i + (d == 0 ? -1 : d == 1 ? 1 : 0);
        int qj = j + (d == 2 ? -1 : d == 3 ? 1 : 0);
        int qk = k + (d == 4 ? -1 : d == 5 ? 1 : 0);
        if (qi < 0 || qi >= p.nx || qj < 0 || qj >= p.ny || qk < 0 || qk >= p.nz) continue;
        CellVals<Chem, T> Q;
        getQ(qi + p.nx * (qj + p.ny * qk), Q);
        T Hg = harm(P.g, Q.g);
        T dPhi = P.phiL - Q.phiL;
        T accL = Make<T>::c(0.0);
#pragma unroll
        for (int m = 0; m < NL; ++m) {
            T dc = P.c[m] - Q.c[m];
            if (!relax) R[m] += Hg * dc * Sc(p.D0[m] * p.h);
            if (p.zc[m] != 0.0) {
                T Hm = harm(P.g * P.c[m], Q.g * Q.c[m]);
                if (!relax) R[m] += Hm * dPhi * Sc(p.kappa_m[m] * p.h);
                accL += Hg * dc * Sc(p.Kd[m]) + Hm * dPhi * Sc(p.Km[m]);
            }
        }
        R[PHIL] += accL * h;
        if (st && Q.ph == 1) R[PHIS] += (P.phiS - Q.phiS) * Sc(p.kappa_s * p.h);
    }

    // ---- reaction sources (structure only)
    if (st) {
        T S[NL], Ss[2], qL, qS;
        sources<Chem, T>(p, P.c, P.es, P.phiL, P.phiS, tH, S, Ss, qL, qS);
        const Sc V = Sc(p.V);
        if (!relax) {
#pragma unroll
            for (int m = 0; m < NL; ++m) R[m] -= S[m] * V;
#pragma unroll
            for (int s = 0; s < NS; ++s) R[NL + s] -= Ss[s] * V;
        }
        R[PHIL] -= qL * V;
        R[PHIS] -= qS * V;
    }
    // ---- anode face x = nx (Eq. 27) and current collector x = 0 (Eq. 25)
    if (i == p.nx - 1) {
        T rA = anode_rate<T>(p, P.c[0], P.phiL);
        if (!relax) R[0] += rA * Sc(p.kAno * p.A);
        R[PHIL] += rA * Sc(p.F * p.kAno * p.A);
    }
    if (i == 0 && st) R[PHIS] += Make<T>::c(p.j_cc * jscale * p.A);
}

// ------------------------------------------------------------------ pass 1: transport factor
template <class Chem, class S, bool TAN>
__device__ __forceinline__ void dg0_g_cell(const DevParams& p, const Geo& g, const S* __restrict__ z,
                                           const S* __restrict__ v, S* __restrict__ gb, S* __restrict__ gbd, int cell) {
    int ph = g.phase[cell];
    int sidx = g.cmap[cell];
    typedef typename std::conditional<TAN, Dual<S>, S>::type T;
    T c[Chem::NL], es[2];
#pragma unroll
    for (int m = 0; m < Chem::NL; ++m) {
        int64_t o = p.off[m] + cell;
        c[m] = Make<T>::var(z[o], TAN ? v[o] : 0.0);
    }
    es[0] = es[1] = Make<T>::c(0.0);
    if (Chem::NS == 2 && ph == 1) {
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            int64_t o = p.off[Chem::NL + s] + sidx;
            es[s] = Make<T>::var(z[o], TAN ? v[o] : 0.0);
        }
    }
    T eL = liquid_fraction<Chem, T>(p, ph, es);
    T gg = transport_factor<Chem, T>(p, eL, c);
    gb[cell] = val(gg);
    if (TAN) {
        if constexpr (TAN) gbd[cell] = gg.d;
    }
}

template <class Chem, class S, bool TAN>
__global__ void __launch_bounds__(128) k_dg0_g(const DevParams p, const Geo g, const S* __restrict__ z,
                                               const S* __restrict__ v, S* __restrict__ gb, S* __restrict__ gbd) {
    int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= p.n_cell) return;
    dg0_g_cell<Chem, S, TAN>(p, g, z, v, gb, gbd, cell);
}

template <class Chem, class S, bool TAN, bool OWN, class T>
__device__ __forceinline__ void load_vals(const DevParams& p, const Geo& g, int cell, const S* z, const S* v,
                                          const S* gb, const S* gbd, int seed, CellVals<Chem, T>& P) {
    P.ph = g.phase[cell];
    P.sidx = g.cmap[cell];
#pragma unroll
    for (int m = 0; m < Chem::NL; ++m) {
        int64_t o = p.off[m] + cell;
        P.c[m] = Make<T>::var(z[o], TAN ? (double)v[o] : (seed == m ? 1.0 : 0.0));
    }
    {
        int64_t o = p.off[Chem::PHIL] + cell;
        P.phiL = Make<T>::var(z[o], TAN ? (double)v[o] : (seed == Chem::PHIL ? 1.0 : 0.0));
    }
    P.es[0] = P.es[1] = Make<T>::c(0.0);
    P.phiS = Make<T>::c(0.0);
    if (P.ph == 1) {
#pragma unroll
        for (int s = 0; s < Chem::NS; ++s) {
            int64_t o = p.off[Chem::NL + s] + P.sidx;
            P.es[s] = Make<T>::var(z[o], TAN ? (double)v[o] : (seed == Chem::NL + s ? 1.0 : 0.0));
        }
        int64_t o = p.off[Chem::PHIS] + P.sidx;
        P.phiS = Make<T>::var(z[o], TAN ? (double)v[o] : (seed == Chem::PHIS ? 1.0 : 0.0));
    }
    if (OWN && seed >= 0) {
        // own transport factor with the seeded direction
        T eL = liquid_fraction<Chem, T>(p, P.ph, P.es);
        P.g = transport_factor<Chem, T>(p, eL, P.c);
    } else {
        P.g = Make<T>::var(gb[cell], TAN ? (double)gbd[cell] : 0.0);
    }
}

// ------------------------------------------------------------------ residual
template <class Chem>
__device__ __forceinline__ void dg0_res_cell(const DevParams& p, const Geo& g, const double* __restrict__ z,
                                             const double* __restrict__ zn, const double* __restrict__ gb,
                                             double t, double dt, int relax, double* __restrict__ r, int cell) {
    int i, j, k;
    cell_ijk(p, cell, i, j, k);
    CellVals<Chem, double> P;
    load_vals<Chem, double, false, true>(p, g, cell, z, z, gb, gb, -1, P);
    double old[Chem::NF];
    const bool st = P.ph == 1;
#pragma unroll
    for (int f = 0; f < Chem::NF; ++f) {
        bool sf = p.is_struct[f];
        old[f] = (!sf) ? zn[p.off[f] + cell] : (st ? zn[p.off[f] + P.sidx] : 0.0);
    }
    auto getQ = [&](int q, CellVals<Chem, double>& Q) { load_vals<Chem, double, false, false>(p, g, q, z, z, gb, gb, -1, Q); };
    double tH = smooth_step(t);
    double R[Chem::NF];
    dg0_cell<Chem, double>(p, i, j, k, P, getQ, old, tH, relax ? tH : 1.0, dt, relax, R);
#pragma unroll
    for (int f = 0; f < Chem::NF; ++f) {
        if (!p.is_struct[f]) r[p.off[f] + cell] = R[f];
        else if (st) r[p.off[f] + P.sidx] = R[f];
    }
}

template <class Chem>
__global__ void __launch_bounds__(128) k_dg0_res(const DevParams p, const Geo g, const double* __restrict__ z,
                                                 const double* __restrict__ zn, const double* __restrict__ gb,
                                                 double t, double dt, int relax, double* __restrict__ r) {
    int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= p.n_cell) return;
    dg0_res_cell<Chem>(p, g, z, zn, gb, t, dt, relax, r, cell);
}

// ------------------------------------------------------------------ Jacobian-vector product
template <class Chem, class S>
__device__ __forceinline__ void dg0_jvp_cell(const DevParams& p, const Geo& g, const S* __restrict__ z,
                                             const S* __restrict__ v, const S* __restrict__ gb,
                                             const S* __restrict__ gbd, double t, double dt, int relax,
                                             double sc_dt, S* __restrict__ out, int cell) {
    typedef Dual<S> T;
    int i, j, k;
    cell_ijk(p, cell, i, j, k);
    CellVals<Chem, T> P;
    load_vals<Chem, S, true, true>(p, g, cell, z, v, gb, gbd, -1, P);
    double old[Chem::NF];
#pragma unroll
    for (int f = 0; f < Chem::NF; ++f) old[f] = 0.0;
    auto getQ = [&](int q, CellVals<Chem, T>& Q) { load_vals<Chem, S, true, false>(p, g, q, z, v, gb, gbd, -1, Q); };
    double tH = smooth_step(t);
    T R[Chem::NF];
    dg0_cell<Chem, T>(p, i, j, k, P, getQ, old, tH, relax ? tH : 1.0, dt, relax, R);
    const bool st = P.ph == 1;
#pragma unroll
    for (int f = 0; f < Chem::NF; ++f) {
        S o = R[f].d;
        if (sc_dt > 0.0) o = o * S(sc_dt * p.rscale[f]);
        if (!p.is_struct[f]) out[p.off[f] + cell] = o;
        else if (st) out[p.off[f] + P.sidx] = o;
    }
}

template <class Chem, class S>
__global__ void __launch_bounds__(128) k_dg0_jvp(const DevParams p, const Geo g, const S* __restrict__ z,
                                                 const S* __restrict__ v, const S* __restrict__ gb,
                                                 const S* __restrict__ gbd, double t, double dt, int relax,
                                                 double sc_dt, S* __restrict__ out) {
    int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= p.n_cell) return;
    dg0_jvp_cell<Chem, S>(p, g, z, v, gb, gbd, t, dt, relax, sc_dt, out, cell);
}

// ------------------------------------------------------------------ diagonal blocks of S J
// blk[cell][row][col] = dt * rscale[row] * dR_row/dz_col over the voxel's own unknowns; rows
// and columns of fields the voxel does not carry are the identity.
template <class Chem, class S>
__global__ void __launch_bounds__(128) k_dg0_blk(const DevParams p, const Geo g, const S* __restrict__ z,
                                                 const S* __restrict__ gb, double t, double dt, int relax,
                                                 double* __restrict__ blk) {
    int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= p.n_cell) return;
    typedef Dual<S> T;
    constexpr int NF = Chem::NF;
    int i, j, k;
    cell_ijk(p, cell, i, j, k);
    double old[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) old[f] = 0.0;
    auto getQ = [&](int q, CellVals<Chem, T>& Q) { load_vals<Chem, S, false, false>(p, g, q, z, z, gb, gb, -1, Q); };
    double tH = smooth_step(t);
    double* B = blk + (int64_t)cell * NF * NF;
    const int ph = g.phase[cell];
#pragma unroll 1
    for (int col = 0; col < NF; ++col) {
        if (p.is_struct[col] && ph != 1) {
            for (int row = 0; row < NF; ++row) B[row * NF + col] = (row == col) ? 1.0 : 0.0;
            continue;
        }
        CellVals<Chem, T> P;
        load_vals<Chem, S, false, true>(p, g, cell, z, z, gb, gb, col, P);
        T R[NF];
        dg0_cell<Chem, T>(p, i, j, k, P, getQ, old, tH, relax ? tH : 1.0, dt, relax, R);
#pragma unroll
        for (int row = 0; row < NF; ++row) {
            double o = (double)R[row].d * dt * p.rscale[row];
            if (p.is_struct[row] && ph != 1) o = (row == col) ? 1.0 : 0.0;
            B[row * NF + col] = o;
        }
    }
}

// ------------------------------------------------------------------ launchers
static inline int nblocks(int64_t n, int bs) { return (int)((n + bs - 1) / bs); }

cudaError_t dg0_residual(const LaunchCtx& L, const DevParams& p, const Geo& g, const double* z, const double* zn,
                         double t, double dt, int relax, double* r, double* gbuf) {
    int nb = nblocks(p.n_cell, 128);
    if (p.nf == 10) {
        k_dg0_g<ChemTO, double, false><<<nb, 128, 0, L.st>>>(p, g, z, z, gbuf, gbuf);
        k_dg0_res<ChemTO><<<nb, 128, 0, L.st>>>(p, g, z, zn, gbuf, t, dt, relax, r);
    } else {
        k_dg0_g<ChemR3, double, false><<<nb, 128, 0, L.st>>>(p, g, z, z, gbuf, gbuf);
        k_dg0_res<ChemR3><<<nb, 128, 0, L.st>>>(p, g, z, zn, gbuf, t, dt, relax, r);
    }
    *L.counter += 2;
    return cudaGetLastError();
}

template <class S>
cudaError_t dg0_jvp(const LaunchCtx& L, const DevParams& p, const Geo& g, const S* z, const S* v, double t,
                    double dt, int relax, double sc_dt, S* out, S* gbuf, S* gbuf_d) {
    int nb = nblocks(p.n_cell, 128);
    if (p.nf == 10) {
        k_dg0_g<ChemTO, S, true><<<nb, 128, 0, L.st>>>(p, g, z, v, gbuf, gbuf_d);
        k_dg0_jvp<ChemTO, S><<<nb, 128, 0, L.st>>>(p, g, z, v, gbuf, gbuf_d, t, dt, relax, sc_dt, out);
    } else {
        k_dg0_g<ChemR3, S, true><<<nb, 128, 0, L.st>>>(p, g, z, v, gbuf, gbuf_d);
        k_dg0_jvp<ChemR3, S><<<nb, 128, 0, L.st>>>(p, g, z, v, gbuf, gbuf_d, t, dt, relax, sc_dt, out);
    }
    *L.counter += 2;
    return cudaGetLastError();
}
template cudaError_t dg0_jvp<double>(const LaunchCtx&, const DevParams&, const Geo&, const double*, const double*,
                                     double, double, int, double, double*, double*, double*);
template cudaError_t dg0_jvp<float>(const LaunchCtx&, const DevParams&, const Geo&, const float*, const float*,
                                    double, double, int, double, float*, float*, float*);

template <class S>
cudaError_t dg0_blocks(const LaunchCtx& L, const DevParams& p, const Geo& g, const S* z, double t, double dt,
                       int relax, double* blk, S* gbuf) {
    int nb = nblocks(p.n_cell, 128);
    if (p.nf == 10) {
        k_dg0_g<ChemTO, S, false><<<nb, 128, 0, L.st>>>(p, g, z, z, gbuf, gbuf);
        k_dg0_blk<ChemTO, S><<<nb, 128, 0, L.st>>>(p, g, z, gbuf, t, dt, relax, blk);
    } else {
        k_dg0_g<ChemR3, S, false><<<nb, 128, 0, L.st>>>(p, g, z, z, gbuf, gbuf);
        k_dg0_blk<ChemR3, S><<<nb, 128, 0, L.st>>>(p, g, z, gbuf, t, dt, relax, blk);
    }
    *L.counter += 2;
    return cudaGetLastError();
}
template cudaError_t dg0_blocks<double>(const LaunchCtx&, const DevParams&, const Geo&, const double*, double, double,
                                        int, double*, double*);
template cudaError_t dg0_blocks<float>(const LaunchCtx&, const DevParams&, const Geo&, const float*, double, double,
                                       int, double*, float*);

cudaError_t dg0_gfactor(const LaunchCtx& L, const DevParams& p, const Geo& g, const double* z, double* gbuf) {
    int nb = nblocks(p.n_cell, 128);
    if (p.nf == 10) k_dg0_g<ChemTO, double, false><<<nb, 128, 0, L.st>>>(p, g, z, z, gbuf, gbuf);
    else k_dg0_g<ChemR3, double, false><<<nb, 128, 0, L.st>>>(p, g, z, z, gbuf, gbuf);
    *L.counter += 1;
    return cudaGetLastError();
}

// ------------------------------------------------------------------ batched instances
// One launch over the voxels of several DG0 instances (each its own grid, parameters and buffers):
// the batch's block range is the concatenation of the instances' ranges, every block belongs to
// one instance (map), and the block copies that instance's job record into shared memory.
// Every voxel goes through the same device functions as in the single-instance kernels, so the
// results are those of the instances run alone.
template <class S>
__device__ __forceinline__ const Job0<S>& stage_job0(const Job0<S>* jobs, const int2* map, Job0<S>* sj) {
    const int j = map[blockIdx.x].x;
    const int4* src = reinterpret_cast<const int4*>(jobs + j);
    int4* dst = reinterpret_cast<int4*>(sj);
    for (int w = threadIdx.x; w < (int)(sizeof(Job0<S>) / 16); w += blockDim.x) dst[w] = src[w];
    __syncthreads();
    return *sj;
}

template <class Chem, class S, bool TAN>
__global__ void k_batch_dg0_g(const Job0<S>* __restrict__ jobs, const int2* __restrict__ map) {
    __shared__ __align__(16) Job0<S> sj;
    const Job0<S>& J = stage_job0(jobs, map, &sj);
    const int cell = map[blockIdx.x].y * blockDim.x + threadIdx.x;
    if (cell >= J.p.n_cell) return;
    dg0_g_cell<Chem, S, TAN>(J.p, J.g, J.z, TAN ? J.v : J.z, J.gb, J.gbd, cell);
}

template <class Chem>
__global__ void k_batch_dg0_res(const Job0<double>* __restrict__ jobs, const int2* __restrict__ map) {
    __shared__ __align__(16) Job0<double> sj;
    const Job0<double>& J = stage_job0(jobs, map, &sj);
    const int cell = map[blockIdx.x].y * blockDim.x + threadIdx.x;
    if (cell >= J.p.n_cell) return;
    dg0_res_cell<Chem>(J.p, J.g, J.z, J.zn, J.gb, J.t, J.dt, J.relax, J.out, cell);
}

template <class Chem, class S>
__global__ void k_batch_dg0_jvp(const Job0<S>* __restrict__ jobs, const int2* __restrict__ map) {
    __shared__ __align__(16) Job0<S> sj;
    const Job0<S>& J = stage_job0(jobs, map, &sj);
    const int cell = map[blockIdx.x].y * blockDim.x + threadIdx.x;
    if (cell >= J.p.n_cell) return;
    dg0_jvp_cell<Chem, S>(J.p, J.g, J.z, J.v, J.gb, J.gbd, J.t, J.dt, J.relax, J.sc_dt, J.out, cell);
}

// mode 0: residual (S = double), 1: Jacobian-vector product; two launches (transport factors, voxels)
template <class S>
cudaError_t dg0_batch(const LaunchCtx& L, bool tradeoff, int mode, const Job0<S>* d_jobs, const int2* d_map,
                      int nblk, int bs) {
    if (nblk <= 0) return cudaSuccess;
    if (mode == 0) {
        if constexpr (std::is_same<S, double>::value) {
            if (tradeoff) {
                k_batch_dg0_g<ChemTO, double, false><<<nblk, bs, 0, L.st>>>(d_jobs, d_map);
                k_batch_dg0_res<ChemTO><<<nblk, bs, 0, L.st>>>(d_jobs, d_map);
            } else {
                k_batch_dg0_g<ChemR3, double, false><<<nblk, bs, 0, L.st>>>(d_jobs, d_map);
                k_batch_dg0_res<ChemR3><<<nblk, bs, 0, L.st>>>(d_jobs, d_map);
            }
        } else {
            return cudaErrorInvalidValue;
        }
    } else if (tradeoff) {
        k_batch_dg0_g<ChemTO, S, true><<<nblk, bs, 0, L.st>>>(d_jobs, d_map);
        k_batch_dg0_jvp<ChemTO, S><<<nblk, bs, 0, L.st>>>(d_jobs, d_map);
    } else {
        k_batch_dg0_g<ChemR3, S, true><<<nblk, bs, 0, L.st>>>(d_jobs, d_map);
        k_batch_dg0_jvp<ChemR3, S><<<nblk, bs, 0, L.st>>>(d_jobs, d_map);
    }
    *L.counter += 2;
    return cudaGetLastError();
}

template <class Chem, class S>
static int max_block_of() {
    cudaFuncAttributes a, b;
    if (cudaFuncGetAttributes(&a, k_batch_dg0_g<Chem, S, true>) != cudaSuccess) return 0;
    if (cudaFuncGetAttributes(&b, k_batch_dg0_jvp<Chem, S>) != cudaSuccess) return 0;
    return std::min(a.maxThreadsPerBlock, b.maxThreadsPerBlock);
}

int dg0_batch_max_block(bool tradeoff, bool f32) {
    if (tradeoff) return f32 ? max_block_of<ChemTO, float>() : max_block_of<ChemTO, double>();
    return f32 ? max_block_of<ChemR3, float>() : max_block_of<ChemR3, double>();
}

template cudaError_t dg0_batch<double>(const LaunchCtx&, bool, int, const Job0<double>*, const int2*, int, int);
template cudaError_t dg0_batch<float>(const LaunchCtx&, bool, int, const Job0<float>*, const int2*, int, int);

}  // namespace dgls
