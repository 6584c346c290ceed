// Linear-algebra kernels of the Newton-GMRES solver: cell-block-Jacobi inversion and
// application, fused multi-vector dot products and updates for classical Gram-Schmidt with
// re-orthogonalisation, scaled norms and the battery reductions (cell voltage, ledger).
//
// Every reduction runs on a fixed grid of RED_BLOCKS x RED_THREADS threads with a fixed
// summation order (per-thread grid-stride partial sums, a shared-memory tree per block, then one
// block summing the per-block partials in index order), so results are bitwise reproducible
// from run to run.
#include "internal.h"

namespace dgls {

static inline int nblocks(int64_t n, int bs) { return (int)((n + bs - 1) / bs); }

// ------------------------------------------------------------------ block Jacobi
// Gauss-Jordan inversion with partial pivoting of one nf x nf block per thread, in place: at step k
// the pivot row is swapped in, column k is replaced by the inverse's column (pivot 1 / a_kk, the
// others -a_ik / a_kk) while the rows are eliminated, and the row swaps are undone at the end by the
// same column swaps in reverse order.  Half the work and local memory of the augmented [A | I] form.
__global__ void k_block_invert(double* __restrict__ blk, int64_t nblk, int nf, float* __restrict__ blk32,
                               int* __restrict__ bad) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nblk) return;
    double a[DG_MAXF][DG_MAXF];
    int rec[DG_MAXF];
    double* B = blk + b * nf * nf;
    for (int r = 0; r < nf; ++r)
        for (int c = 0; c < nf; ++c) a[r][c] = B[r * nf + c];
    bool singular = false;
    for (int k = 0; k < nf; ++k) {
        int piv = k;
        double best = fabs(a[k][k]);
        for (int r = k + 1; r < nf; ++r)
            if (fabs(a[r][k]) > best) { best = fabs(a[r][k]); piv = r; }
        if (!(best > 0.0) || !isfinite(best)) { singular = true; break; }
        rec[k] = piv;
        if (piv != k)
            for (int c = 0; c < nf; ++c) { double t = a[k][c]; a[k][c] = a[piv][c]; a[piv][c] = t; }
        const double d = 1.0 / a[k][k];
        a[k][k] = 1.0;
        for (int c = 0; c < nf; ++c) a[k][c] *= d;
        for (int r = 0; r < nf; ++r) {
            if (r == k) continue;
            const double f = a[r][k];
            if (f == 0.0) continue;
            a[r][k] = 0.0;
            for (int c = 0; c < nf; ++c) a[r][c] -= f * a[k][c];
        }
    }
    if (singular) {
        atomicAdd(bad, 1);
        for (int r = 0; r < nf; ++r)
            for (int c = 0; c < nf; ++c) a[r][c] = (r == c) ? 1.0 : 0.0;
    } else {
        for (int k = nf - 1; k >= 0; --k)
            if (rec[k] != k)
                for (int r = 0; r < nf; ++r) { double t = a[r][k]; a[r][k] = a[r][rec[k]]; a[r][rec[k]] = t; }
    }
    for (int r = 0; r < nf; ++r)
        for (int c = 0; c < nf; ++c) {
            B[r * nf + c] = a[r][c];
            if (blk32) blk32[(int64_t)(r * nf + c) * nblk + b] = (float)a[r][c];   // entry-major: coalesced apply
        }
}

cudaError_t block_invert(const LaunchCtx& L, double* blk, int64_t nblk, int nf, float* blk32, int* bad) {
    k_block_invert<<<nblocks(nblk, 64), 64, 0, L.st>>>(blk, nblk, nf, blk32, bad);
    *L.counter += 1;
    return cudaGetLastError();
}

// out = B^{-1} v per block; DG0: one block per voxel, DG1: one block per (node, voxel).
template <class S, class BT, int NF>
__global__ void __launch_bounds__(128) k_block_apply(const DevParams p, const Geo g, const BT* __restrict__ blk,
                                                     const S* __restrict__ v, S* __restrict__ out) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int nn = p.order == 1 ? 8 : 1;
    if (b >= (int64_t)p.n_cell * nn) return;
    int node = (int)(b / p.n_cell);
    int cell = (int)(b - (int64_t)node * p.n_cell);
    int ph = g.phase[cell];
    int sidx = g.cmap[cell];
    int64_t idx[NF];
    S x[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        if (!p.is_struct[f]) idx[f] = p.off[f] + (int64_t)node * p.flen[f] + cell;
        else idx[f] = (ph == 1) ? p.off[f] + (int64_t)node * p.flen[f] + sidx : -1;
        x[f] = idx[f] >= 0 ? v[idx[f]] : S(0);
    }
    // FP64 blocks: NF x NF consecutive per block; FP32 blocks: entry-major, [r * NF + c][block]
    const bool soa = std::is_same<BT, float>::value;
    const int64_t nblk = (int64_t)p.n_cell * nn;
    const BT* B = soa ? blk + b : blk + b * NF * NF;
    const int64_t es = soa ? nblk : 1;
#pragma unroll
    for (int r = 0; r < NF; ++r) {
        if (idx[r] < 0) continue;
        S acc = S(0);
#pragma unroll
        for (int c = 0; c < NF; ++c) acc += S(B[(int64_t)(r * NF + c) * es]) * x[c];
        out[idx[r]] = acc;
    }
}

template <class S>
cudaError_t block_apply(const LaunchCtx& L, const DevParams& p, const Geo& g, const void* blk, const S* v, S* out) {
    int64_t n = (int64_t)p.n_cell * (p.order == 1 ? 8 : 1);
    int nb = nblocks(n, 128);
    typedef typename std::conditional<std::is_same<S, float>::value, float, double>::type BT;
    if (p.nf == 10) k_block_apply<S, BT, 10><<<nb, 128, 0, L.st>>>(p, g, (const BT*)blk, v, out);
    else k_block_apply<S, BT, 5><<<nb, 128, 0, L.st>>>(p, g, (const BT*)blk, v, out);
    *L.counter += 1;
    return cudaGetLastError();
}
template cudaError_t block_apply<double>(const LaunchCtx&, const DevParams&, const Geo&, const void*, const double*, double*);
template cudaError_t block_apply<float>(const LaunchCtx&, const DevParams&, const Geo&, const void*, const float*, float*);

// ------------------------------------------------------------------ reductions
__device__ __forceinline__ double block_sum(double v, double* sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    double r = sh[0];
    __syncthreads();
    return r;
}

// partial[k][block] -> out[k], summed in block order by one block per k
__global__ void k_finish(const double* __restrict__ partial, int nparts, int k, double* __restrict__ out) {
    __shared__ double sh[RED_THREADS];
    for (int v = blockIdx.x; v < k; v += gridDim.x) {
        double acc = 0.0;
        for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc += partial[(int64_t)v * nparts + i];
        double s = block_sum(acc, sh);
        if (threadIdx.x == 0) out[v] = s;
    }
}

// h[v] = sum_i V[v][i] w[i] for v < k, one pass over w and the k basis vectors.
// With SELF, h[k] = sum_i w[i]^2 as well (the norm that the re-orthogonalisation test needs).
template <class S, int KM, bool SELF>
__global__ void __launch_bounds__(RED_THREADS) k_mdot(const S* __restrict__ V, int64_t ld, int64_t n, int k,
                                                      const S* __restrict__ w, double* __restrict__ partial) {
    __shared__ double sh[RED_THREADS];
    // per-thread partial sums in the basis precision (FP32 FMAs for an FP32 basis: on GB300 an
    // FP64 FMA per 4-byte element would make this pass FP64-bound), block and grid sums in FP64
    S acc[KM + 1];
#pragma unroll
    for (int v = 0; v <= KM; ++v) acc[v] = S(0);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        S wi = w[i];
#pragma unroll
        for (int v = 0; v < KM; ++v) acc[v] += V[(int64_t)v * ld + i] * wi;
        if (SELF) acc[KM] += wi * wi;
    }
#pragma unroll
    for (int v = 0; v < KM + (SELF ? 1 : 0); ++v) {
        double s = block_sum((double)acc[v], sh);
        if (threadIdx.x == 0) partial[(int64_t)v * gridDim.x + blockIdx.x] = s;
    }
}

// launch k_mdot instantiated for exactly k vectors: a larger bucket would issue the predicated-off
// FMAs of the unused accumulators, which on GB300's FP64 pipe costs as much as the real ones
template <class S, int K, bool SELF>
static void mdot_launch(const LaunchCtx& L, const S* V, int64_t ld, int64_t n, int k, const S* w, double* partial) {
    if constexpr (K <= MAXK) {
        if (k == K) {
            k_mdot<S, K, SELF><<<RED_BLOCKS, RED_THREADS, 0, L.st>>>(V, ld, n, k, w, partial);
            return;
        }
        mdot_launch<S, K + 1, SELF>(L, V, ld, n, k, w, partial);
    }
}

template <class S>
cudaError_t mdot(const LaunchCtx& L, const S* V, int64_t ld, int64_t n, int k, const S* w, double* partial,
                 double* out, bool self) {
    if (k < 1 || k > MAXK) return cudaErrorInvalidValue;
    if (self) mdot_launch<S, 1, true>(L, V, ld, n, k, w, partial);
    else mdot_launch<S, 1, false>(L, V, ld, n, k, w, partial);
    const int nk = k + (self ? 1 : 0);
    k_finish<<<nk < 32 ? nk : 32, RED_THREADS, 0, L.st>>>(partial, RED_BLOCKS, nk, out);
    *L.counter += 2;
    return cudaGetLastError();
}
template cudaError_t mdot<double>(const LaunchCtx&, const double*, int64_t, int64_t, int, const double*, double*, double*,
                                  bool);
template cudaError_t mdot<float>(const LaunchCtx&, const float*, int64_t, int64_t, int, const float*, double*, double*,
                                 bool);

// w += sign * sum_v h[v] V[v]
template <class S>
__global__ void __launch_bounds__(256) k_maxpy(S* __restrict__ w, const S* __restrict__ V, int64_t ld, int64_t n, int k,
                                               const double* __restrict__ h, double sign) {
    __shared__ S hs[MAXK];
    if (threadIdx.x < k) hs[threadIdx.x] = (S)(sign * h[threadIdx.x]);
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        S acc = w[i];
        for (int v = 0; v < k; ++v) acc += hs[v] * V[(int64_t)v * ld + i];
        w[i] = acc;
    }
}

template <class S>
cudaError_t maxpy(const LaunchCtx& L, S* w, const S* V, int64_t ld, int64_t n, int k, const double* h, double sign) {
    k_maxpy<S><<<RED_BLOCKS * 2, 256, 0, L.st>>>(w, V, ld, n, k, h, sign);
    *L.counter += 1;
    return cudaGetLastError();
}
template cudaError_t maxpy<double>(const LaunchCtx&, double*, const double*, int64_t, int64_t, int, const double*, double);
template cudaError_t maxpy<float>(const LaunchCtx&, float*, const float*, int64_t, int64_t, int, const double*, double);

// w -= sum_v h[v] V[v] and nrm2 = sum_i w[i]^2 of the updated vector, in one pass (fixed grid).
template <class S>
__global__ void __launch_bounds__(RED_THREADS) k_maxpy_norm(S* __restrict__ w, const S* __restrict__ V, int64_t ld,
                                                            int64_t n, int k, const double* __restrict__ h,
                                                            double* __restrict__ partial) {
    __shared__ S hs[MAXK];
    __shared__ double sh[RED_THREADS];
    if (threadIdx.x < k) hs[threadIdx.x] = (S)(-h[threadIdx.x]);
    __syncthreads();
    S nrm = S(0);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        S acc = w[i];
        for (int v = 0; v < k; ++v) acc += hs[v] * V[(int64_t)v * ld + i];
        w[i] = acc;
        nrm += acc * acc;
    }
    double s = block_sum((double)nrm, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

template <class S>
cudaError_t maxpy_norm(const LaunchCtx& L, S* w, const S* V, int64_t ld, int64_t n, int k, const double* h,
                       double* partial, double* nrm2) {
    if (k < 1 || k > MAXK) return cudaErrorInvalidValue;
    k_maxpy_norm<S><<<RED_BLOCKS, RED_THREADS, 0, L.st>>>(w, V, ld, n, k, h, partial);
    k_finish<<<1, RED_THREADS, 0, L.st>>>(partial, RED_BLOCKS, 1, nrm2);
    *L.counter += 2;
    return cudaGetLastError();
}
template cudaError_t maxpy_norm<double>(const LaunchCtx&, double*, const double*, int64_t, int64_t, int, const double*,
                                        double*, double*);
template cudaError_t maxpy_norm<float>(const LaunchCtx&, float*, const float*, int64_t, int64_t, int, const double*,
                                       double*, double*);

// dst = a * src / sqrt(*nrm2_dev) (nrm2_dev holds a squared norm) or dst = a * src if nrm2_dev is null
template <class S>
__global__ void k_scale_copy(S* __restrict__ dst, const S* __restrict__ src, int64_t n, const double* __restrict__ nrm2,
                             double a) {
    double f = a;
    if (nrm2) f = a / sqrt(*nrm2);
    const S fs = (S)f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i] * fs;
}

template <class S>
cudaError_t scale_copy(const LaunchCtx& L, S* dst, const S* src, int64_t n, const double* nrm2, double a) {
    k_scale_copy<S><<<RED_BLOCKS * 2, 256, 0, L.st>>>(dst, src, n, nrm2, a);
    *L.counter += 1;
    return cudaGetLastError();
}
template cudaError_t scale_copy<double>(const LaunchCtx&, double*, const double*, int64_t, const double*, double);
template cudaError_t scale_copy<float>(const LaunchCtx&, float*, const float*, int64_t, const double*, double);

// out = -(dt * rscale[field]) r  (the scaled right-hand side of the Newton system)
template <class S>
__global__ void k_neg_scaled(const DevParams p, const double* __restrict__ r, double dt, S* __restrict__ out) {
    for (int f = 0; f < p.nf; ++f) {
        int64_t len = p.flen[f] * (p.order == 1 ? 8 : 1);
        double s = -dt * p.rscale[f];
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
            out[p.off[f] + i] = (S)(s * r[p.off[f] + i]);
    }
}
template <class S>
cudaError_t neg_scaled(const LaunchCtx& L, const DevParams& p, const double* r, double dt, S* out) {
    k_neg_scaled<S><<<RED_BLOCKS * 2, 256, 0, L.st>>>(p, r, dt, out);
    *L.counter += 1;
    return cudaGetLastError();
}
template cudaError_t neg_scaled<double>(const LaunchCtx&, const DevParams&, const double*, double, double*);
template cudaError_t neg_scaled<float>(const LaunchCtx&, const DevParams&, const double*, double, float*);

// sum_i (dt * rscale[field(i)] * r_i)^2
__global__ void __launch_bounds__(RED_THREADS) k_scaled_norm2(const DevParams p, const double* __restrict__ r, double dt,
                                                              double* __restrict__ partial) {
    __shared__ double sh[RED_THREADS];
    double acc = 0.0;
    for (int f = 0; f < p.nf; ++f) {
        int64_t len = p.flen[f] * (p.order == 1 ? 8 : 1);
        double s = dt * p.rscale[f];
        const double* x = r + p.off[f];
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
            double y = s * x[i];
            acc += y * y;
        }
    }
    double s = block_sum(acc, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

cudaError_t scaled_norm2(const LaunchCtx& L, const DevParams& p, const double* r, double dt, double* partial, double* out) {
    k_scaled_norm2<<<RED_BLOCKS, RED_THREADS, 0, L.st>>>(p, r, dt, partial);
    k_finish<<<1, RED_THREADS, 0, L.st>>>(partial, RED_BLOCKS, 1, out);
    *L.counter += 2;
    return cudaGetLastError();
}

__global__ void k_sum(const double* __restrict__ x, int64_t n, double* __restrict__ partial) {
    __shared__ double sh[RED_THREADS];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) acc += x[i];
    double s = block_sum(acc, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

cudaError_t reduce_sum(const LaunchCtx& L, const double* x, int64_t n, double* partial, double* out) {
    k_sum<<<RED_BLOCKS, RED_THREADS, 0, L.st>>>(x, n, partial);
    k_finish<<<1, RED_THREADS, 0, L.st>>>(partial, RED_BLOCKS, 1, out);
    *L.counter += 2;
    return cudaGetLastError();
}

// ------------------------------------------------------------------ elementwise
__global__ void k_axpby(double* __restrict__ y, double a, const double* __restrict__ x, double b, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = a * y[i] + b * x[i];
}
cudaError_t axpby(const LaunchCtx& L, double* y, double a, const double* x, double b, int64_t n) {
    k_axpby<<<RED_BLOCKS * 2, 256, 0, L.st>>>(y, a, x, b, n);
    *L.counter += 1;
    return cudaGetLastError();
}

template <class S>
__global__ void k_saxpby(S* __restrict__ y, double a, const S* __restrict__ x, double b, int64_t n) {
    const S as = (S)a, bs = (S)b;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = as * y[i] + bs * x[i];
}
template <class S>
cudaError_t saxpby(const LaunchCtx& L, S* y, double a, const S* x, double b, int64_t n) {
    k_saxpby<S><<<RED_BLOCKS * 2, 256, 0, L.st>>>(y, a, x, b, n);
    *L.counter += 1;
    return cudaGetLastError();
}
template cudaError_t saxpby<double>(const LaunchCtx&, double*, double, const double*, double, int64_t);
template cudaError_t saxpby<float>(const LaunchCtx&, float*, double, const float*, double, int64_t);

__global__ void k_to_f32(float* __restrict__ d, const double* __restrict__ s, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        d[i] = (float)s[i];
}
cudaError_t to_f32(const LaunchCtx& L, float* dst, const double* src, int64_t n) {
    k_to_f32<<<RED_BLOCKS * 2, 256, 0, L.st>>>(dst, src, n);
    *L.counter += 1;
    return cudaGetLastError();
}

__global__ void k_to_f64_add(double* __restrict__ d, const float* __restrict__ s, double a, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        d[i] = a * d[i] + (double)s[i];
}
cudaError_t to_f64_add(const LaunchCtx& L, double* dst, const float* src, double a, int64_t n) {
    k_to_f64_add<<<RED_BLOCKS * 2, 256, 0, L.st>>>(dst, src, a, n);
    *L.counter += 1;
    return cudaGetLastError();
}

__global__ void k_row_scales(const DevParams p, double dt, double* __restrict__ s) {
    for (int f = 0; f < p.nf; ++f) {
        int64_t len = p.flen[f] * (p.order == 1 ? 8 : 1);
        double v = dt * p.rscale[f];
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
            s[p.off[f] + i] = v;
    }
}
cudaError_t row_scales(const LaunchCtx& L, const DevParams& p, double dt, double* s) {
    k_row_scales<<<RED_BLOCKS, 256, 0, L.st>>>(p, dt, s);
    *L.counter += 1;
    return cudaGetLastError();
}

__global__ void k_fill(const DevParams p, const double* __restrict__ vals, double* __restrict__ z) {
    for (int f = 0; f < p.nf; ++f) {
        int64_t len = p.flen[f] * (p.order == 1 ? 8 : 1);
        double v = vals[f];
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
            z[p.off[f] + i] = v;
    }
}
cudaError_t fill_equilibrium(const LaunchCtx& L, const DevParams& p, const double* vals, double* z) {
    k_fill<<<RED_BLOCKS, 256, 0, L.st>>>(p, vals, z);
    *L.counter += 1;
    return cudaGetLastError();
}

// ------------------------------------------------------------------ battery quantities
// U_cell (Eq. A1): mean over the structure faces at x = 0 of Phi^S (DG0: the voxel value;
// DG1: the trace at xi = -1 at the 2 x 2 face Gauss points).
__global__ void __launch_bounds__(RED_THREADS) k_cc_sum(const DevParams p, const Geo g, const double* __restrict__ z,
                                                        double* __restrict__ partial) {
    __shared__ double sh[RED_THREADS];
    double acc = 0.0, cnt = 0.0;
    const int fS = p.nf - 1;
    const double al = 0.5 * (1.0 + sqrt(3.0)), be = 0.5 * (1.0 - sqrt(3.0));
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < (int64_t)p.ny * p.nz; q += (int64_t)gridDim.x * blockDim.x) {
        int cell = (int)(q * p.nx);
        if (g.phase[cell] != 1) continue;
        int s = g.cmap[cell];
        cnt += 1.0;
        if (p.order == 0) {
            acc += z[p.off[fS] + s];
        } else {
            double fsum = 0.0;
            for (int bc = 0; bc < 4; ++bc) {      // (b, c) face point
                int n0 = 0 + 2 * (bc & 1) + 4 * (bc >> 1);
                double v0 = z[p.off[fS] + (int64_t)n0 * p.flen[fS] + s];
                double v1 = z[p.off[fS] + (int64_t)(n0 + 1) * p.flen[fS] + s];
                fsum += al * v0 + be * v1;
            }
            acc += 0.25 * fsum;
        }
    }
    double s1 = block_sum(acc, sh);
    double s2 = block_sum(cnt, sh);
    if (threadIdx.x == 0) { partial[blockIdx.x] = s1; partial[gridDim.x + blockIdx.x] = s2; }
}

__global__ void k_div(double* out) { out[0] = out[0] / out[1]; }

cudaError_t cell_voltage(const LaunchCtx& L, const DevParams& p, const Geo& g, const double* z, double* partial, double* out) {
    k_cc_sum<<<RED_BLOCKS, RED_THREADS, 0, L.st>>>(p, g, z, partial);
    k_finish<<<2, RED_THREADS, 0, L.st>>>(partial, RED_BLOCKS, 2, out);
    k_div<<<1, 1, 0, L.st>>>(out);
    *L.counter += 3;
    return cudaGetLastError();
}

// Ledger totals: sulfur, lithium (mol), liquid charge (C), Phi^L face means at x = nx and x = 0.
template <class Chem>
__global__ void __launch_bounds__(RED_THREADS) k_ledger(const DevParams p, const Geo g, const double* __restrict__ z,
                                                        double* __restrict__ partial) {
    __shared__ double sh[RED_THREADS];
    double aS = 0.0, aLi = 0.0, aQ = 0.0, aA = 0.0, a0 = 0.0;
    const int nn = p.order == 1 ? 8 : 1;
    const double M = p.order == 1 ? p.V / 8.0 : p.V;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < (int64_t)p.n_cell * nn; b += (int64_t)gridDim.x * blockDim.x) {
        int node = (int)(b / p.n_cell);
        int cell = (int)(b - (int64_t)node * p.n_cell);
        int ph = g.phase[cell];
        int s = g.cmap[cell];
        double c[Chem::NL], es[2] = {0.0, 0.0};
        for (int m = 0; m < Chem::NL; ++m) c[m] = z[p.off[m] + (int64_t)node * p.flen[m] + cell];
        if (Chem::NS == 2 && ph == 1)
            for (int q = 0; q < 2; ++q) es[q] = z[p.off[Chem::NL + q] + (int64_t)node * p.flen[Chem::NL + q] + s];
        double eL = val(liquid_fraction<Chem, double>(p, ph, es));
        double sS = 0.0, q = 0.0;
        for (int m = 0; m < Chem::NL; ++m) { sS += p.wS[m] * c[m]; q += p.zc[m] * c[m]; }
        aS += M * eL * sS;
        aLi += M * eL * c[0];
        aQ += M * eL * p.F * q;
        if (Chem::NS == 2 && ph == 1) {
            aS += M * (8.0 * p.rhoM[0] * es[0] + p.rhoM[1] * es[1]);
            aLi += M * 2.0 * p.rhoM[1] * es[1];
        }
        int i = cell % p.nx;
        const int a = node & 1;
        double phiL = z[p.off[Chem::PHIL] + (int64_t)node * p.flen[Chem::PHIL] + cell];
        if (p.order == 0) {
            if (i == p.nx - 1) aA += phiL;
            if (i == 0) a0 += phiL;
        } else {
            const double al = 0.5 * (1.0 + sqrt(3.0)), be = 0.5 * (1.0 - sqrt(3.0));
            if (i == p.nx - 1) aA += 0.25 * (a == 1 ? al : be) * phiL;
            if (i == 0) a0 += 0.25 * (a == 0 ? al : be) * phiL;
        }
    }
    double v[5] = {aS, aLi, aQ, aA, a0};
    for (int k = 0; k < 5; ++k) {
        double s = block_sum(v[k], sh);
        if (threadIdx.x == 0) partial[(int64_t)k * gridDim.x + blockIdx.x] = s;
    }
}

__global__ void k_ledger_norm(const DevParams p, double* out) {
    double nf = (double)p.ny * p.nz;
    out[3] /= nf;
    out[4] /= nf;
}

cudaError_t ledger(const LaunchCtx& L, const DevParams& p, const Geo& g, const double* z, double* partial, double* out5) {
    if (p.nf == 10) k_ledger<ChemTO><<<RED_BLOCKS, RED_THREADS, 0, L.st>>>(p, g, z, partial);
    else k_ledger<ChemR3><<<RED_BLOCKS, RED_THREADS, 0, L.st>>>(p, g, z, partial);
    k_finish<<<5, RED_THREADS, 0, L.st>>>(partial, RED_BLOCKS, 5, out5);
    k_ledger_norm<<<1, 1, 0, L.st>>>(p, out5);
    *L.counter += 3;
    return cudaGetLastError();
}

// FP64 -> FP32 copies of several vectors in one launch: launch block b converts elements
// [map[b].y * CONV_BLOCK_ELEMS, +CONV_BLOCK_ELEMS) of vector map[b].x
__global__ void __launch_bounds__(256) k_to_f32_batched(const ConvJob* __restrict__ jobs, const int2* __restrict__ map) {
    const ConvJob J = jobs[map[blockIdx.x].x];
    const int64_t base = (int64_t)map[blockIdx.x].y * CONV_BLOCK_ELEMS;
    for (int e = threadIdx.x; e < CONV_BLOCK_ELEMS; e += blockDim.x) {
        const int64_t i = base + e;
        if (i < J.n) J.dst[i] = (float)J.src[i];
    }
}

cudaError_t to_f32_batched(const LaunchCtx& L, const ConvJob* d_jobs, const int2* d_map, int nblk) {
    if (nblk <= 0) return cudaSuccess;
    k_to_f32_batched<<<nblk, 256, 0, L.st>>>(d_jobs, d_map);
    *L.counter += 1;
    return cudaGetLastError();
}

}  // namespace dgls
