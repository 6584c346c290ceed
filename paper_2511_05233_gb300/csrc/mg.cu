// Two-stage (CPR-type) preconditioner of the Newton systems: an aggregation multigrid for the
// potential block, followed by cell-block Jacobi on the whole system.
//
// The two charge equations of Tab. 4 carry no storage term, so their block of S J is elliptic:
// with the Butler-Volmer derivatives (a = -M dq_S/dPhi^S >= 0) it is exactly
//   (A x)_L = sum_faces G_L (x_L,P - x_L,Q) + a (x_L - x_S) + d_L x_L
//   (A x)_S = sum_faces G_S (x_S,P - x_S,Q) + a (x_S - x_L) + d_S x_S
// a symmetric M-matrix (two coupled graph Laplacians grounded by the anode exchange current d_L),
// where G_L = h sum_j K^m_j {g c_j}_H (DG0) is the liquid conductance of the migration terms and
// G_S = h kappa_S the solid one.  Block Jacobi alone needs O(n) Krylov iterations on it; one
// V-cycle of this multigrid removes the smooth potential error at every level.
//
// DG1 uses the same operator on voxel averages: with the voxel-constant prolongation P, P^T A P of
// the DG1 potential block keeps only the penalty term of Eq. 46 (face conductance
// penalty (h/4) sum_{4 face points} sum_j K^m_j {g c_j}_H) and the node sums of a and d.
//
// Hierarchy: 2 x 2 x 2 aggregation with piecewise-constant interpolation (the Galerkin coarse
// operator of a graph Laplacian is the aggregated graph Laplacian: coarse conductances are sums of
// the fine conductances crossing aggregate boundaries); damped 2 x 2 block-Jacobi smoothing;
// the coarsest level (<= 64 voxels) is solved exactly with a dense inverse.
#include <cstring>
#include <type_traits>
#include <vector>

#include "internal.h"

namespace dgls {

namespace {
constexpr double SQ3 = 1.7320508075688772935;
constexpr double ALPHA = 0.5 * (1.0 + SQ3);
constexpr double BETA = 0.5 * (1.0 - SQ3);

inline int nb(int64_t n, int bs) { return (int)((n + bs - 1) / bs); }

__device__ __forceinline__ void ijk(int c, int nx, int ny, int& i, int& j, int& k) {
    i = c % nx;
    int r = c / nx;
    j = r % ny;
    k = r / ny;
}
}  // namespace

// ------------------------------------------------------------------ level-0 coefficients (DG0)
template <class Chem>
__global__ void k_pp_dg0(const DevParams p, const Geo g, const double* __restrict__ z, const double* __restrict__ gb,
                         double t, double dt, int relax, MGLevel L) {
    int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= p.n_cell) return;
    constexpr int NL = Chem::NL;
    const double s = dt * p.rscale[Chem::PHIL];
    int i, j, k;
    ijk(cell, p.nx, p.ny, i, j, k);
    const int ph = g.phase[cell];
    const int sidx = g.cmap[cell];
    const bool st = ph == 1;
    double cP[NL];
    for (int m = 0; m < NL; ++m) cP[m] = z[p.off[m] + cell];
    const double gP = gb[cell];
    for (int d = 0; d < 3; ++d) {
        int qi = i + (d == 0), qj = j + (d == 1), qk = k + (d == 2);
        double gl = 0.0, gs = 0.0;
        if (qi < p.nx && qj < p.ny && qk < p.nz) {
            int q = qi + p.nx * (qj + p.ny * qk);
            double gQ = gb[q];
            for (int m = 0; m < NL; ++m)
                if (p.zc[m] != 0.0) gl += p.Km[m] * harm(gP * cP[m], gQ * z[p.off[m] + q]);
            gl *= p.h;
            if (st && g.phase[q] == 1) gs = p.h * p.kappa_s;
        }
        L.gL[(int64_t)d * L.n + cell] = s * gl;
        L.gS[(int64_t)d * L.n + cell] = s * gs;
    }
    double a = 0.0, dL = 0.0, dS = 0.0;
    if (st) {
        typedef Dual<double> T;
        T c[NL], es[2], Sv[NL], Ss[2], qL, qS;
        for (int m = 0; m < NL; ++m) c[m] = mkd(cP[m], 0.0);
        es[0] = es[1] = mkd(0.0, 0.0);
        for (int q = 0; q < Chem::NS; ++q) es[q] = mkd(z[p.off[NL + q] + sidx], 0.0);
        T phiL = mkd(z[p.off[Chem::PHIL] + cell], 0.0);
        T phiS = mkd(z[p.off[Chem::PHIS] + sidx], 1.0);
        sources<Chem, T>(p, c, es, phiL, phiS, smooth_step(t), Sv, Ss, qL, qS);
        a = -p.V * qS.d;
    }
    if (i == p.nx - 1) {
        Dual<double> r = anode_rate<Dual<double>>(p, mkd(cP[0], 0.0), mkd(z[p.off[Chem::PHIL] + cell], 1.0));
        dL = p.A * p.F * p.kAno * r.d;
    }
    if (relax) {
        dL += p.V / dt;
        if (st) dS += p.V / dt;
    }
    L.a[cell] = s * a;
    L.dL[cell] = s * dL;
    L.dS[cell] = s * dS;
    L.st[cell] = st ? 1 : 0;
}

// ------------------------------------------------------------------ level-0 coefficients (DG1)
template <class Chem>
__global__ void k_pp_dg1(const DevParams p, const Geo g, const double* __restrict__ z, const double* __restrict__ gb,
                         double t, double dt, int relax, MGLevel L) {
    int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= p.n_cell) return;
    constexpr int NL = Chem::NL;
    const double s = dt * p.rscale[Chem::PHIL];         // node row scale of the potential rows
    int i, j, k;
    ijk(cell, p.nx, p.ny, i, j, k);
    const int ph = g.phase[cell];
    const int sidx = g.cmap[cell];
    const bool st = ph == 1;
    auto zf = [&](int f, int n, int idx) { return z[p.off[f] + (int64_t)n * p.flen[f] + idx]; };
    const double wf = 0.25 * p.h * p.h;
    for (int d = 0; d < 3; ++d) {
        int qi = i + (d == 0), qj = j + (d == 1), qk = k + (d == 2);
        double gl = 0.0, gs = 0.0;
        if (qi < p.nx && qj < p.ny && qk < p.nz) {
            int q = qi + p.nx * (qj + p.ny * qk);
            for (int pt = 0; pt < 4; ++pt) {
                int u = pt & 1, w = pt >> 1;
                int n0, n1;
                if (d == 0) { n0 = 0 + 2 * u + 4 * w; n1 = n0 + 1; }
                else if (d == 1) { n0 = u + 0 + 4 * w; n1 = n0 + 2; }
                else { n0 = u + 2 * w; n1 = n0 + 4; }
                // own + face point (slot 8 + (2d+1)*4 + pt), neighbour - face point (slot 8 + 2d*4 + pt)
                double gP = gb[(int64_t)(8 + (2 * d + 1) * 4 + pt) * p.n_cell + cell];
                double gQ = gb[(int64_t)(8 + (2 * d) * 4 + pt) * p.n_cell + q];
                double acc = 0.0;
                for (int m = 0; m < NL; ++m) {
                    if (p.zc[m] == 0.0) continue;
                    double cp = ALPHA * zf(m, n1, cell) + BETA * zf(m, n0, cell);
                    double cq = ALPHA * zf(m, n0, q) + BETA * zf(m, n1, q);
                    acc += p.Km[m] * harm(gP * cp, gQ * cq);
                }
                gl += acc;
            }
            gl *= wf * p.penalty / p.h;
            if (st && g.phase[q] == 1) gs = 4.0 * wf * p.penalty / p.h * p.kappa_s;
        }
        L.gL[(int64_t)d * L.n + cell] = s * gl;
        L.gS[(int64_t)d * L.n + cell] = s * gs;
    }
    double a = 0.0, dL = 0.0, dS = 0.0;
    const double M = p.V / 8.0;
    if (st) {
        typedef Dual<double> T;
        for (int n = 0; n < 8; ++n) {
            T c[NL], es[2], Sv[NL], Ss[2], qL, qS;
            for (int m = 0; m < NL; ++m) c[m] = mkd(zf(m, n, cell), 0.0);
            es[0] = es[1] = mkd(0.0, 0.0);
            for (int q = 0; q < Chem::NS; ++q) es[q] = mkd(zf(NL + q, n, sidx), 0.0);
            T phiL = mkd(zf(Chem::PHIL, n, cell), 0.0);
            T phiS = mkd(zf(Chem::PHIS, n, sidx), 1.0);
            sources<Chem, T>(p, c, es, phiL, phiS, smooth_step(t), Sv, Ss, qL, qS);
            a += -M * qS.d;
        }
    }
    if (i == p.nx - 1) {
        for (int pt = 0; pt < 4; ++pt) {
            int n0 = 2 * (pt & 1) + 4 * (pt >> 1), n1 = n0 + 1;
            double cLi = ALPHA * zf(0, n1, cell) + BETA * zf(0, n0, cell);
            double phL = ALPHA * zf(Chem::PHIL, n1, cell) + BETA * zf(Chem::PHIL, n0, cell);
            Dual<double> r = anode_rate<Dual<double>>(p, mkd(cLi, 0.0), mkd(phL, 1.0));
            dL += wf * p.F * p.kAno * r.d;
        }
    }
    if (relax) {
        dL += p.V / dt;
        if (st) dS += p.V / dt;
    }
    L.a[cell] = s * a;
    L.dL[cell] = s * dL;
    L.dS[cell] = s * dS;
    L.st[cell] = st ? 1 : 0;
}

// ------------------------------------------------------------------ hierarchy
__global__ void k_mg_coarsen(MGLevel F, MGLevel C) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C.n) return;
    int I, J, K;
    ijk(c, C.nx, C.ny, I, J, K);
    double gl[3] = {0, 0, 0}, gs[3] = {0, 0, 0}, a = 0, dL = 0, dS = 0;
    int st = 0;
    for (int dk = 0; dk < 2; ++dk)
        for (int dj = 0; dj < 2; ++dj)
            for (int di = 0; di < 2; ++di) {
                int i = 2 * I + di, j = 2 * J + dj, k = 2 * K + dk;
                if (i >= F.nx || j >= F.ny || k >= F.nz) continue;
                int f = i + F.nx * (j + F.ny * k);
                a += F.a[f];
                dL += F.dL[f];
                dS += F.dS[f];
                st |= F.st[f];
                // faces leaving the aggregate in + direction come from its last child layer
                if (di == 1) { gl[0] += F.gL[f]; gs[0] += F.gS[f]; }
                if (dj == 1) { gl[1] += F.gL[(int64_t)F.n + f]; gs[1] += F.gS[(int64_t)F.n + f]; }
                if (dk == 1) { gl[2] += F.gL[2 * (int64_t)F.n + f]; gs[2] += F.gS[2 * (int64_t)F.n + f]; }
            }
    // an aggregate with a single child layer along d has no "+" child: its + faces are those of
    // that layer (only at the grid end, where they are zero anyway)
    for (int d = 0; d < 3; ++d) {
        C.gL[(int64_t)d * C.n + c] = gl[d];
        C.gS[(int64_t)d * C.n + c] = gs[d];
    }
    C.a[c] = a;
    C.dL[c] = dL;
    C.dS[c] = dS;
    C.st[c] = st;
}

// 2 x 2 block diagonal of A and its inverse
__global__ void k_mg_diag(MGLevel L) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= L.n) return;
    int i, j, k;
    ijk(c, L.nx, L.ny, i, j, k);
    double sl = 0.0, ss = 0.0;
    for (int d = 0; d < 3; ++d) {
        sl += L.gL[(int64_t)d * L.n + c];
        ss += L.gS[(int64_t)d * L.n + c];
    }
    if (i > 0) { sl += L.gL[c - 1]; ss += L.gS[c - 1]; }
    if (j > 0) { sl += L.gL[(int64_t)L.n + c - L.nx]; ss += L.gS[(int64_t)L.n + c - L.nx]; }
    if (k > 0) { sl += L.gL[2 * (int64_t)L.n + c - L.nx * L.ny]; ss += L.gS[2 * (int64_t)L.n + c - L.nx * L.ny]; }
    double a = L.a[c];
    double d00 = sl + a + L.dL[c], d01 = -a, d10 = -a, d11 = ss + a + L.dS[c];
    if (!L.st[c]) { d01 = d10 = 0.0; d11 = 1.0; }
    if (!(d00 > 0.0)) d00 = 1.0;
    if (!(d11 > 0.0)) d11 = 1.0;
    double det = d00 * d11 - d01 * d10;
    L.dinv[c] = d11 / det;
    L.dinv[(int64_t)L.n + c] = -d01 / det;
    L.dinv[2 * (int64_t)L.n + c] = -d10 / det;
    L.dinv[3 * (int64_t)L.n + c] = d00 / det;
}

// (A x) at cell c for both fields
__device__ __forceinline__ void apply_A(const MGLevel& L, const double* x, int c, double& yl, double& ys) {
    int i, j, k;
    ijk(c, L.nx, L.ny, i, j, k);
    const int64_t n = L.n;
    double xl = x[c], xs = x[n + c];
    double accl = 0.0, accs = 0.0;
    // + neighbours
    if (i + 1 < L.nx) { double gl = L.gL[c], gs = L.gS[c]; accl += gl * (xl - x[c + 1]); accs += gs * (xs - x[n + c + 1]); }
    if (j + 1 < L.ny) { double gl = L.gL[n + c], gs = L.gS[n + c]; int q = c + L.nx; accl += gl * (xl - x[q]); accs += gs * (xs - x[n + q]); }
    if (k + 1 < L.nz) { double gl = L.gL[2 * n + c], gs = L.gS[2 * n + c]; int q = c + L.nx * L.ny; accl += gl * (xl - x[q]); accs += gs * (xs - x[n + q]); }
    // - neighbours
    if (i > 0) { int q = c - 1; accl += L.gL[q] * (xl - x[q]); accs += L.gS[q] * (xs - x[n + q]); }
    if (j > 0) { int q = c - L.nx; accl += L.gL[n + q] * (xl - x[q]); accs += L.gS[n + q] * (xs - x[n + q]); }
    if (k > 0) { int q = c - L.nx * L.ny; accl += L.gL[2 * n + q] * (xl - x[q]); accs += L.gS[2 * n + q] * (xs - x[n + q]); }
    double a = L.a[c];
    yl = accl + a * (xl - xs) + L.dL[c] * xl;
    ys = L.st[c] ? accs + a * (xs - xl) + L.dS[c] * xs : xs;
}

// x_out = x_in + w D^-1 (b - A x_in); zero_in: x_in = 0
__global__ void k_mg_jacobi(MGLevel L, const double* __restrict__ xin, double* __restrict__ xout, double w, int zero_in) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= L.n) return;
    const int64_t n = L.n;
    double rl = L.b[c], rs = L.b[n + c];
    double xl = 0.0, xs = 0.0;
    if (!zero_in) {
        double yl, ys;
        apply_A(L, xin, c, yl, ys);
        rl -= yl;
        rs -= ys;
        xl = xin[c];
        xs = xin[n + c];
    }
    xout[c] = xl + w * (L.dinv[c] * rl + L.dinv[n + c] * rs);
    xout[n + c] = xs + w * (L.dinv[2 * n + c] * rl + L.dinv[3 * n + c] * rs);
}

// coarse b = restriction of the fine residual b - A x (sum over the aggregate; S only over
// structure children)
__global__ void k_mg_restrict(MGLevel F, MGLevel C) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C.n) return;
    int I, J, K;
    ijk(c, C.nx, C.ny, I, J, K);
    double bl = 0.0, bs = 0.0;
    for (int dk = 0; dk < 2; ++dk)
        for (int dj = 0; dj < 2; ++dj)
            for (int di = 0; di < 2; ++di) {
                int i = 2 * I + di, j = 2 * J + dj, k = 2 * K + dk;
                if (i >= F.nx || j >= F.ny || k >= F.nz) continue;
                int f = i + F.nx * (j + F.ny * k);
                double yl, ys;
                apply_A(F, F.x, f, yl, ys);
                bl += F.b[f] - yl;
                if (F.st[f]) bs += F.b[(int64_t)F.n + f] - ys;
            }
    C.b[c] = bl;
    C.b[(int64_t)C.n + c] = bs;
}

__global__ void k_mg_prolong(MGLevel F, MGLevel C) {
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F.n) return;
    int i, j, k;
    ijk(f, F.nx, F.ny, i, j, k);
    int c = (i >> 1) + C.nx * ((j >> 1) + C.ny * (k >> 1));
    F.x[f] += C.x[c];
    if (F.st[f]) F.x[(int64_t)F.n + f] += C.x[(int64_t)C.n + c];
}

// coarsest level (n <= 64 voxels, m = 2n <= 128 unknowns): dense inverse at set-up by in-place
// Gauss-Jordan elimination in shared memory (m x m doubles, at most 128 KB) in one thread block of
// 1024 threads.  A connected, grounded operator is a symmetric M-matrix and needs no pivoting, but
// the structure can hold parts that are neither: a voxel whose Phi^S has no structure neighbour and
// no surface left (a_V = 0) has an empty row, and a cluster that nothing grounds is singular.  So a
// row whose diagonal is not positive becomes an identity row, and a pivot that has lost all but
// rounding of its row's diagonal leaves its unknown out of the coarse correction (row and column of
// the inverse set to zero) instead of dividing by it.  One dense matrix-vector product per V-cycle.
constexpr int DENSE_THREADS = 1024;
constexpr int DENSE_MAX = 128;

__global__ void __launch_bounds__(DENSE_THREADS) k_mg_dense_build(MGLevel L) {
    extern __shared__ double A[];            // [m][m] row-major: L fields 0..n-1, S fields n..2n-1
    __shared__ double rowk[DENSE_MAX], colk[DENSE_MAX], diag0[DENSE_MAX];
    const int m = 2 * L.n;
    const int tid = threadIdx.x;
    for (int e = tid; e < m * m; e += DENSE_THREADS) A[e] = 0.0;
    __syncthreads();
    if (tid < m) {
        const int r = tid;
        const int cell = r < L.n ? r : r - L.n;
        const bool isL = r < L.n;
        int i, j, k;
        ijk(cell, L.nx, L.ny, i, j, k);
        const int64_t n = L.n;
        const double* G = isL ? L.gL : L.gS;
        double* row = A + (int64_t)r * m;
        double diag = 0.0;
        auto nbr = [&](int q, double g) {
            if (g == 0.0) return;
            diag += g;
            row[isL ? q : n + q] -= g;
        };
        if (i + 1 < L.nx) nbr(cell + 1, G[cell]);
        if (j + 1 < L.ny) nbr(cell + L.nx, G[n + cell]);
        if (k + 1 < L.nz) nbr(cell + L.nx * L.ny, G[2 * n + cell]);
        if (i > 0) nbr(cell - 1, G[cell - 1]);
        if (j > 0) nbr(cell - L.nx, G[n + cell - L.nx]);
        if (k > 0) nbr(cell - L.nx * L.ny, G[2 * n + cell - L.nx * L.ny]);
        const double a = L.a[cell];
        if (isL) {
            row[r] += diag + a + L.dL[cell];
            row[n + cell] -= a;
        } else if (L.st[cell]) {
            row[r] += diag + a + L.dS[cell];
            row[cell] -= a;
        } else {
            for (int c = 0; c < m; ++c) row[c] = 0.0;
            row[r] = 1.0;
        }
        // an empty row (no conductance, no coupling, no diagonal term) has an empty column too
        // (the operator is symmetric): make it an identity row
        if (!(row[r] > 0.0)) {
            for (int c = 0; c < m; ++c) row[c] = 0.0;
            row[r] = 1.0;
        }
        diag0[r] = row[r];
    }
    __syncthreads();
    // pivot k: row k <- row k / p (entry k <- 1/p); row i != k <- row i - A[i][k] row k (entry k <- -A[i][k]/p)
    for (int kk = 0; kk < m; ++kk) {
        if (tid < m) {
            const double piv = A[(int64_t)kk * m + kk];
            const double pinv = (piv > 1e-14 * diag0[kk]) ? 1.0 / piv : 0.0;
            rowk[tid] = tid == kk ? pinv : A[(int64_t)kk * m + tid] * pinv;
            colk[tid] = A[(int64_t)tid * m + kk];
        }
        __syncthreads();
        for (int e = tid; e < m * m; e += DENSE_THREADS) {
            const int i = e / m, c = e - i * m;
            if (i == kk) A[e] = rowk[c];
            else if (c == kk) A[e] = -colk[i] * rowk[kk];
            else A[e] -= colk[i] * rowk[c];
        }
        __syncthreads();
    }
    for (int e = tid; e < m * m; e += DENSE_THREADS) L.dense[e] = A[e];
}

__global__ void __launch_bounds__(128) k_mg_dense_solve(MGLevel L) {
    const int m = 2 * L.n;
    const int r = threadIdx.x;
    if (r >= m) return;
    const double* A = L.dense + (int64_t)r * m;
    double acc = 0.0;
    for (int c = 0; c < m; ++c) acc += A[c] * L.b[c];
    L.x[r] = acc;
}

// ------------------------------------------------------------------ CPR restriction / prolongation
template <class S>
__global__ void k_cpr_restrict(const DevParams p, const Geo g, const S* __restrict__ v, MGLevel L) {
    int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= p.n_cell) return;
    const int nn = p.order == 1 ? 8 : 1;
    const int fL = p.nf - 2, fS = p.nf - 1;
    const int s = g.cmap[cell];
    double bl = 0.0, bs = 0.0;
    for (int n = 0; n < nn; ++n) {
        bl += (double)v[p.off[fL] + (int64_t)n * p.flen[fL] + cell];
        if (s >= 0) bs += (double)v[p.off[fS] + (int64_t)n * p.flen[fS] + s];
    }
    L.b[cell] = bl;
    L.b[(int64_t)L.n + cell] = bs;
}

// y = P x (potential fields), zero elsewhere
template <class S>
__global__ void k_cpr_prolong(const DevParams p, const Geo g, MGLevel L, S* __restrict__ y) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int nn = p.order == 1 ? 8 : 1;
    if (b >= (int64_t)p.n_cell * nn) return;
    const int n = (int)(b / p.n_cell);
    const int cell = (int)(b - (int64_t)n * p.n_cell);
    const int fL = p.nf - 2, fS = p.nf - 1;
    for (int f = 0; f < fL; ++f) {
        if (!p.is_struct[f]) y[p.off[f] + (int64_t)n * p.flen[f] + cell] = S(0);
        else if (g.cmap[cell] >= 0) y[p.off[f] + (int64_t)n * p.flen[f] + g.cmap[cell]] = S(0);
    }
    y[p.off[fL] + (int64_t)n * p.flen[fL] + cell] = (S)L.x[cell];
    const int s = g.cmap[cell];
    if (s >= 0) y[p.off[fS] + (int64_t)n * p.flen[fS] + s] = (S)L.x[(int64_t)L.n + cell];
}

// ------------------------------------------------------------------ species coarse level
// At large dt the rows of a liquid species are dominated by diffusion, whose smooth error the node
// blocks cannot remove.  With the voxel-constant prolongation P, P^T (S J) P of species m keeps,
// of Eqs. 45-47, the node terms and the interior penalty only (the volume integral and the
// consistency term of Eq. 46 act on gradients, which vanish on voxel constants):
//   (A x)_P = sum_faces G (x_P - x_Q) + d_P x_P
//   G   = dt rscale_m (h^2/4) (penalty/h) D_m^0 sum_{4 face points} H(g_P, g_Q)
//   d_P = dt rscale_m sum_{8 nodes} dR_m/dc_m   (storage and own-species reaction derivative),
// plus, for Li+, the derivative of the anode exchange (Eq. 27) on the x = nx face.  Migration and
// the couplings to the other species and to the potentials are left to the node blocks.  Two
// species share one hierarchy as its two fields, uncoupled (a = 0, every voxel carries both; a
// missing second species is an identity row).
template <class Chem, class SJ>
__global__ void k_sp_dg1(const DevParams p, const Geo g, const double* __restrict__ z, const double* __restrict__ gb,
                         const SJ* __restrict__ jn, double dt, double mdt, int m0, int m1, MGLevel L) {
    int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= p.n_cell) return;
    constexpr int NF = Chem::NF;
    int i, j, k;
    ijk(cell, p.nx, p.ny, i, j, k);
    const int ph = g.phase[cell];
    const double s = dt * p.rscale[m0];                 // all liquid species rows share one scale
    const double wf = 0.25 * p.h * p.h;
    const double gpen = s * wf * p.penalty / p.h;
    const double D0 = p.D0[m0], D1 = m1 >= 0 ? p.D0[m1] : 0.0;
    for (int d = 0; d < 3; ++d) {
        int qi = i + (d == 0), qj = j + (d == 1), qk = k + (d == 2);
        double hs = 0.0;
        if (qi < p.nx && qj < p.ny && qk < p.nz) {
            int q = qi + p.nx * (qj + p.ny * qk);
            for (int pt = 0; pt < 4; ++pt) {
                // own + face point (slot 8 + (2d+1)*4 + pt), neighbour - face point (slot 8 + 2d*4 + pt)
                double gP = gb[(int64_t)(8 + (2 * d + 1) * 4 + pt) * p.n_cell + cell];
                double gQ = gb[(int64_t)(8 + (2 * d) * 4 + pt) * p.n_cell + q];
                hs += harm(gP, gQ);
            }
        }
        L.gL[(int64_t)d * L.n + cell] = gpen * D0 * hs;
        L.gS[(int64_t)d * L.n + cell] = gpen * D1 * hs;
    }
    double d0 = 0.0, d1 = 0.0;
    if (ph == 1) {
        const int sidx = g.cmap[cell];
        for (int n = 0; n < 8; ++n) {
            const SJ* J = jn + (int64_t)n * NF * NF * p.n_struct + sidx;
            d0 += (double)J[(int64_t)(m0 * NF + m0) * p.n_struct];
            if (m1 >= 0) d1 += (double)J[(int64_t)(m1 * NF + m1) * p.n_struct];
        }
    } else {   // storage alone: eps_L M / dt per node (eps_L = 1 in pores, the separator porosity there)
        d0 = 8.0 * mdt * (ph == 2 ? p.eps_sep : 1.0);
        d1 = m1 >= 0 ? d0 : 0.0;
    }
    if (m0 == 0 && i == p.nx - 1) {
        for (int pt = 0; pt < 4; ++pt) {
            int n0 = 2 * (pt & 1) + 4 * (pt >> 1), n1 = n0 + 1;
            double cLi = ALPHA * z[p.off[0] + (int64_t)n1 * p.flen[0] + cell] + BETA * z[p.off[0] + (int64_t)n0 * p.flen[0] + cell];
            double phL = ALPHA * z[p.off[Chem::PHIL] + (int64_t)n1 * p.flen[Chem::PHIL] + cell] +
                         BETA * z[p.off[Chem::PHIL] + (int64_t)n0 * p.flen[Chem::PHIL] + cell];
            Dual<double> r = anode_rate<Dual<double>>(p, mkd(cLi, 1.0), mkd(phL, 0.0));
            d0 += wf * p.kAno * r.d;
        }
    }
    L.a[cell] = 0.0;
    L.dL[cell] = s * d0;
    L.dS[cell] = s * d1;
    L.st[cell] = m1 >= 0 ? 1 : 0;
}

// DG0: the species block of S J itself (P = identity): conductance dt rscale_m h D_m^0 H(g_P, g_Q)
// (Eq. 48), diagonal dt rscale_m (V eps_L / dt - V dS_m/dc_m), and the anode exchange for Li+.
template <class Chem>
__global__ void k_sp_dg0(const DevParams p, const Geo g, const double* __restrict__ z, const double* __restrict__ gb,
                         double t, double dt, int m0, int m1, MGLevel L) {
    int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= p.n_cell) return;
    constexpr int NL = Chem::NL;
    int i, j, k;
    ijk(cell, p.nx, p.ny, i, j, k);
    const int ph = g.phase[cell];
    const int sidx = g.cmap[cell];
    const double s = dt * p.rscale[m0];
    const double D0 = p.D0[m0], D1 = m1 >= 0 ? p.D0[m1] : 0.0;
    const double gP = gb[cell];
    for (int d = 0; d < 3; ++d) {
        int qi = i + (d == 0), qj = j + (d == 1), qk = k + (d == 2);
        double hg = 0.0;
        if (qi < p.nx && qj < p.ny && qk < p.nz) hg = s * p.h * harm(gP, gb[qi + p.nx * (qj + p.ny * qk)]);
        L.gL[(int64_t)d * L.n + cell] = hg * D0;
        L.gS[(int64_t)d * L.n + cell] = hg * D1;
    }
    double es[2] = {0.0, 0.0};
    if (ph == 1)
        for (int q = 0; q < Chem::NS; ++q) es[q] = z[p.off[NL + q] + sidx];
    const double vdt = p.V / dt * liquid_fraction<Chem, double>(p, ph, es);
    double d0 = vdt, d1 = m1 >= 0 ? vdt : 0.0;
    if (ph == 1) {
        typedef Dual<double> T;
        for (int w = 0; w < 2; ++w) {
            const int m = w == 0 ? m0 : m1;
            if (m < 0) continue;
            T c[NL], e2[2], Sv[NL], Ss[2], qL, qS;
            for (int l = 0; l < NL; ++l) c[l] = mkd(z[p.off[l] + cell], l == m ? 1.0 : 0.0);
            e2[0] = mkd(es[0], 0.0);
            e2[1] = mkd(es[1], 0.0);
            T phiL = mkd(z[p.off[Chem::PHIL] + cell], 0.0);
            T phiS = mkd(z[p.off[Chem::PHIS] + sidx], 0.0);
            sources<Chem, T>(p, c, e2, phiL, phiS, smooth_step(t), Sv, Ss, qL, qS);
            (w == 0 ? d0 : d1) += -p.V * Sv[m].d;
        }
    }
    if (m0 == 0 && i == p.nx - 1) {
        Dual<double> r = anode_rate<Dual<double>>(p, mkd(z[p.off[0] + cell], 1.0), mkd(z[p.off[Chem::PHIL] + cell], 0.0));
        d0 += p.A * p.kAno * r.d;
    }
    L.a[cell] = 0.0;
    L.dL[cell] = s * d0;
    L.dS[cell] = s * d1;
    L.st[cell] = m1 >= 0 ? 1 : 0;
}

// b = P^T v of the pair's two species (sum over the nodes of the voxel: 8 for DG1, 1 for DG0)
template <class S>
__global__ void k_sp_restrict(const DevParams p, const S* __restrict__ v, int m0, int m1, MGLevel L) {
    int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= p.n_cell) return;
    const int nn = p.order == 1 ? 8 : 1;
    double b0 = 0.0, b1 = 0.0;
    for (int n = 0; n < nn; ++n) {
        b0 += (double)v[p.off[m0] + (int64_t)n * p.flen[m0] + cell];
        if (m1 >= 0) b1 += (double)v[p.off[m1] + (int64_t)n * p.flen[m1] + cell];
    }
    L.b[cell] = b0;
    L.b[(int64_t)L.n + cell] = b1;
}

// y += P x on the pair's two species
template <class S>
__global__ void k_sp_prolong_add(const DevParams p, MGLevel L, int m0, int m1, S* __restrict__ y) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= (int64_t)p.n_cell * (p.order == 1 ? 8 : 1)) return;
    const int n = (int)(b / p.n_cell);
    const int cell = (int)(b - (int64_t)n * p.n_cell);
    y[p.off[m0] + (int64_t)n * p.flen[m0] + cell] += (S)L.x[cell];
    if (m1 >= 0) y[p.off[m1] + (int64_t)n * p.flen[m1] + cell] += (S)L.x[(int64_t)L.n + cell];
}

// ------------------------------------------------------------------ host drivers
cudaError_t mg_levels_alloc(std::vector<MGLevel>& lv, int nx, int ny, int nz, std::vector<void*>& allocs,
                            int64_t* bytes, DevArena* arena) {
    lv.clear();
    int x = nx, y = ny, zz = nz;
    for (;;) {
        MGLevel L;
        std::memset(&L, 0, sizeof(L));
        L.nx = x; L.ny = y; L.nz = zz;
        L.n = x * y * zz;
        auto al = [&](auto** ptr, int64_t cnt) -> cudaError_t {
            void* q = nullptr;
            const bool from_arena = arena && arena->active;
            cudaError_t e = from_arena ? arena_alloc(arena, (size_t)cnt * sizeof(**ptr), &q)
                                       : cudaMalloc(&q, (size_t)cnt * sizeof(**ptr));
            if (e != cudaSuccess) return e;
            if (!from_arena) allocs.push_back(q);
            *bytes += cnt * (int64_t)sizeof(**ptr);
            *ptr = (std::remove_reference_t<decltype(*ptr)>)q;
            return cudaSuccess;
        };
        cudaError_t e;
        if ((e = al(&L.gL, 3 * (int64_t)L.n)) != cudaSuccess) return e;
        if ((e = al(&L.gS, 3 * (int64_t)L.n)) != cudaSuccess) return e;
        if ((e = al(&L.a, L.n)) != cudaSuccess) return e;
        if ((e = al(&L.dL, L.n)) != cudaSuccess) return e;
        if ((e = al(&L.dS, L.n)) != cudaSuccess) return e;
        if ((e = al(&L.st, L.n)) != cudaSuccess) return e;
        if ((e = al(&L.dinv, 4 * (int64_t)L.n)) != cudaSuccess) return e;
        if ((e = al(&L.x, 2 * (int64_t)L.n)) != cudaSuccess) return e;
        if ((e = al(&L.xt, 2 * (int64_t)L.n)) != cudaSuccess) return e;
        if ((e = al(&L.b, 2 * (int64_t)L.n)) != cudaSuccess) return e;
        const bool last = L.n <= 64 || (x == 1 && y == 1 && zz == 1);
        if (last && (e = al(&L.dense, (int64_t)(2 * L.n) * (2 * L.n))) != cudaSuccess) return e;
        lv.push_back(L);
        if (last) break;
        x = (x + 1) / 2;
        y = (y + 1) / 2;
        zz = (zz + 1) / 2;
    }
    return cudaSuccess;
}

// coarse levels, 2 x 2 block diagonals and the dense coarsest inverse of a hierarchy whose level 0
// has just been written
static cudaError_t mg_hierarchy(const LaunchCtx& Lc, std::vector<MGLevel>& lv) {
    for (size_t l = 0; l + 1 < lv.size(); ++l) {
        k_mg_coarsen<<<nb(lv[l + 1].n, 256), 256, 0, Lc.st>>>(lv[l], lv[l + 1]);
        *Lc.counter += 1;
    }
    for (auto& L : lv) {
        k_mg_diag<<<nb(L.n, 256), 256, 0, Lc.st>>>(L);
        *Lc.counter += 1;
    }
    const int m = 2 * lv.back().n;
    const size_t smem = (size_t)m * m * sizeof(double);
    // opt in to more than 48 KB of dynamic shared memory; the attribute belongs to the current
    // device, so it is set on every build (a host call, cheap next to the build itself)
    const cudaError_t attr = cudaFuncSetAttribute(k_mg_dense_build, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  DENSE_MAX * DENSE_MAX * (int)sizeof(double));
    if (attr != cudaSuccess) return attr;
    k_mg_dense_build<<<1, DENSE_THREADS, smem, Lc.st>>>(lv.back());
    *Lc.counter += 1;
    return cudaGetLastError();
}

cudaError_t mg_setup(const LaunchCtx& Lc, const DevParams& p, const Geo& g, const double* z, const double* gb,
                     double t, double dt, int relax, std::vector<MGLevel>& lv) {
    if (lv.empty()) return cudaErrorInvalidValue;
    if (p.order == 0) {
        if (p.nf == 10) k_pp_dg0<ChemTO><<<nb(p.n_cell, 128), 128, 0, Lc.st>>>(p, g, z, gb, t, dt, relax, lv[0]);
        else k_pp_dg0<ChemR3><<<nb(p.n_cell, 128), 128, 0, Lc.st>>>(p, g, z, gb, t, dt, relax, lv[0]);
    } else {
        if (p.nf == 10) k_pp_dg1<ChemTO><<<nb(p.n_cell, 128), 128, 0, Lc.st>>>(p, g, z, gb, t, dt, relax, lv[0]);
        else k_pp_dg1<ChemR3><<<nb(p.n_cell, 128), 128, 0, Lc.st>>>(p, g, z, gb, t, dt, relax, lv[0]);
    }
    *Lc.counter += 1;
    return mg_hierarchy(Lc, lv);
}

// One V-cycle on level l.  warm: start from the current x of level l (a repeated cycle on the finest
// level); otherwise from zero (the first cycle, and every coarse level, which solves for a correction).
static void vcycle(const LaunchCtx& Lc, std::vector<MGLevel>& lv, size_t l, bool warm = false) {
    MGLevel& L = lv[l];
    const double w = 0.8;
    if (l + 1 == lv.size()) {
        k_mg_dense_solve<<<1, 128, 0, Lc.st>>>(L);   // exact: a warm start changes nothing
        *Lc.counter += 1;
        return;
    }
    const int g = nb(L.n, 256);
    k_mg_jacobi<<<g, 256, 0, Lc.st>>>(L, L.x, L.xt, w, warm ? 0 : 1);
    k_mg_jacobi<<<g, 256, 0, Lc.st>>>(L, L.xt, L.x, w, 0);
    k_mg_restrict<<<nb(lv[l + 1].n, 256), 256, 0, Lc.st>>>(L, lv[l + 1]);
    *Lc.counter += 3;
    vcycle(Lc, lv, l + 1);
    k_mg_prolong<<<g, 256, 0, Lc.st>>>(L, lv[l + 1]);
    k_mg_jacobi<<<g, 256, 0, Lc.st>>>(L, L.x, L.xt, w, 0);
    k_mg_jacobi<<<g, 256, 0, Lc.st>>>(L, L.xt, L.x, w, 0);
    *Lc.counter += 3;
}

// y = P (V-cycles on R v): the potential correction of the first CPR stage
template <class S>
cudaError_t cpr_stage1(const LaunchCtx& Lc, const DevParams& p, const Geo& g, std::vector<MGLevel>& lv, int cycles,
                       const S* v, S* y) {
    MGLevel& L0 = lv[0];
    k_cpr_restrict<S><<<nb(p.n_cell, 256), 256, 0, Lc.st>>>(p, g, v, L0);
    *Lc.counter += 1;
    for (int c = 0; c < cycles; ++c) vcycle(Lc, lv, 0, c > 0);
    const int nn = p.order == 1 ? 8 : 1;
    k_cpr_prolong<S><<<nb((int64_t)p.n_cell * nn, 256), 256, 0, Lc.st>>>(p, g, L0, y);
    *Lc.counter += 1;
    return cudaGetLastError();
}
template cudaError_t cpr_stage1<double>(const LaunchCtx&, const DevParams&, const Geo&, std::vector<MGLevel>&, int,
                                        const double*, double*);
template cudaError_t cpr_stage1<float>(const LaunchCtx&, const DevParams&, const Geo&, std::vector<MGLevel>&, int,
                                       const float*, float*);

cudaError_t mg_species_setup(const LaunchCtx& Lc, const DevParams& p, const Geo& g, const double* z, const double* gb,
                             const void* jn, bool jn_f32, double t, double dt, std::vector<MGLevel>* lv, int npairs) {
    if (p.order == 1 && !jn) return cudaErrorInvalidValue;
    const double mdt = (p.V / 8.0) / dt;
    for (int k = 0; k < npairs; ++k) {
        if (lv[k].empty()) return cudaErrorInvalidValue;
        const int m0 = 2 * k, m1 = 2 * k + 1 < p.nl ? 2 * k + 1 : -1;
        const int grid = nb(p.n_cell, 128);
        if (p.order == 0) {
            if (p.nf == 10) k_sp_dg0<ChemTO><<<grid, 128, 0, Lc.st>>>(p, g, z, gb, t, dt, m0, m1, lv[k][0]);
            else k_sp_dg0<ChemR3><<<grid, 128, 0, Lc.st>>>(p, g, z, gb, t, dt, m0, m1, lv[k][0]);
        } else if (p.nf == 10) {
            if (jn_f32) k_sp_dg1<ChemTO, float><<<grid, 128, 0, Lc.st>>>(p, g, z, gb, (const float*)jn, dt, mdt, m0, m1, lv[k][0]);
            else k_sp_dg1<ChemTO, double><<<grid, 128, 0, Lc.st>>>(p, g, z, gb, (const double*)jn, dt, mdt, m0, m1, lv[k][0]);
        } else {
            if (jn_f32) k_sp_dg1<ChemR3, float><<<grid, 128, 0, Lc.st>>>(p, g, z, gb, (const float*)jn, dt, mdt, m0, m1, lv[k][0]);
            else k_sp_dg1<ChemR3, double><<<grid, 128, 0, Lc.st>>>(p, g, z, gb, (const double*)jn, dt, mdt, m0, m1, lv[k][0]);
        }
        *Lc.counter += 1;
        cudaError_t e = mg_hierarchy(Lc, lv[k]);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

// y += sum over the pairs of P V-cycle(P^T v) on the species of each pair
template <class S>
cudaError_t mg_species_apply(const LaunchCtx& Lc, const DevParams& p, std::vector<MGLevel>* lv, int npairs, const S* v,
                             S* y) {
    for (int k = 0; k < npairs; ++k) {
        const int m0 = 2 * k, m1 = 2 * k + 1 < p.nl ? 2 * k + 1 : -1;
        k_sp_restrict<S><<<nb(p.n_cell, 256), 256, 0, Lc.st>>>(p, v, m0, m1, lv[k][0]);
        *Lc.counter += 1;
        vcycle(Lc, lv[k], 0);
        k_sp_prolong_add<S><<<nb((int64_t)p.n_cell * (p.order == 1 ? 8 : 1), 256), 256, 0, Lc.st>>>(p, lv[k][0], m0, m1, y);
        *Lc.counter += 1;
    }
    return cudaGetLastError();
}
template cudaError_t mg_species_apply<double>(const LaunchCtx&, const DevParams&, std::vector<MGLevel>*, int,
                                              const double*, double*);
template cudaError_t mg_species_apply<float>(const LaunchCtx&, const DevParams&, std::vector<MGLevel>*, int,
                                             const float*, float*);

}  // namespace dgls
