// Internal interfaces between the C-ABI layer (api.cu) and the kernel translation units.
#pragma once
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

#include "common.cuh"

namespace dgls {

// Device geometry shared by all kernels.
struct Geo {
    const uint8_t* phase;      // [n_cell]
    const int32_t* cmap;       // [n_cell] structure index or -1
    const int32_t* sidx;       // [n_struct] structure index -> voxel
};

// One level of the potential multigrid (two fields per voxel: Phi^L, Phi^S).
struct MGLevel {
    int nx, ny, nz, n;
    double* gL;    // [3][n] liquid conductance to the + neighbour in x, y, z
    double* gS;    // [3][n] solid conductance to the + neighbour
    double* a;     // [n] Butler-Volmer coupling between the two potentials
    double* dL;    // [n] diagonal of the Phi^L row (anode exchange, relaxation term)
    double* dS;    // [n] diagonal of the Phi^S row (relaxation term)
    uint8_t* st;   // [n] voxel carries Phi^S
    double* dinv;  // [4][n] inverse of the 2 x 2 diagonal block
    double* x;     // [2][n]
    double* xt;    // [2][n]
    double* b;     // [2][n]
    double* dense; // coarsest level only: [2n][4n] Gauss-Jordan workspace, right half = A^{-1}
};

// Workspace carved from one caller-owned device buffer instead of cudaMalloc (a server keeps such
// buffers and reuses them across requests); with base == nullptr the allocations are only counted,
// which sizes the buffer exactly.  Every allocation starts on a 256-byte boundary.
struct DevArena {
    char* base = nullptr;
    int64_t size = 0;
    int64_t used = 0;
    bool active = false;
};
inline cudaError_t arena_alloc(DevArena* a, size_t bytes, void** p) {
    const int64_t off = (a->used + 255) / 256 * 256;
    if (a->base && off + (int64_t)bytes > a->size) return cudaErrorMemoryAllocation;
    *p = a->base ? (void*)(a->base + off) : (void*)(uintptr_t)(off + 256);   // counting: a distinct dummy address
    a->used = off + (int64_t)bytes;
    return cudaSuccess;
}

// Launch counter increment hook (owned by the context).
struct LaunchCtx {
    cudaStream_t st;
    int64_t* counter;
};

// ------------------------------------------------------------------ DG0 (dg0.cu)
// relax: 1 for the parabolic relaxation residual (Sec. 2.8); tH = T_H(t) for the smoothed
// reactions and the ramped current; scale: multiply outputs by dt * rscale (Newton rows).
cudaError_t dg0_residual(const LaunchCtx& L, const DevParams& p, const Geo& g, const double* z,
                         const double* zn, double t, double dt, int relax, double* r, double* gbuf);
template <class S>
cudaError_t dg0_jvp(const LaunchCtx& L, const DevParams& p, const Geo& g, const S* z, const S* v,
                    double t, double dt, int relax, double out_scale_dt, S* out, S* gbuf, S* gbuf_d);
template <class S>
cudaError_t dg0_blocks(const LaunchCtx& L, const DevParams& p, const Geo& g, const S* z,
                       double t, double dt, int relax, double* blk, S* gbuf);
cudaError_t dg0_gfactor(const LaunchCtx& L, const DevParams& p, const Geo& g, const double* z, double* gbuf);

// ------------------------------------------------------------------ DG1 (dg1.cu)
cudaError_t dg1_residual(const LaunchCtx& L, const DevParams& p, const Geo& g, const double* z,
                         const double* zn, double t, double dt, int relax, double* r, double* fbuf, double* flux);
template <class S>
cudaError_t dg1_jvp(const LaunchCtx& L, const DevParams& p, const Geo& g, const S* z, const S* v,
                    double t, double dt, int relax, double out_scale_dt, S* out, S* fbuf, S* fbuf_d);
cudaError_t dg1_gfactor(const LaunchCtx& L, const DevParams& p, const Geo& g, const double* z, double* fbuf);
int64_t dg1_face_buffer_len(const DevParams& p);
// Linearised FP64 DG1 JVP: cached derivative data at a fixed linearisation point.
struct DG1Lin {
    bool f32 = false;       // linearisation stored in FP32 for the FP32 product (mixed precision)
    double* jn = nullptr;   // [8][NF*NF][n_struct] node Jacobians of the structure voxels
    double* gam = nullptr;  // [32][n_cell] 3/(2 eps_L) per transport-factor slot
    double* face = nullptr; // [12][NFD][n_cell] face data of the + faces
    double* gb = nullptr;   // [32][n_cell] transport factors at the linearisation point (FP64 mode)
    double* gbd = nullptr;  // [32][n_cell] their tangents (apply scratch)
    double* flux = nullptr; // [4][NL+2][n_cell] face-flux tangents of one direction (apply scratch)
    float *jn32 = nullptr, *gam32 = nullptr, *face32 = nullptr, *gb32 = nullptr, *gbd32 = nullptr, *flux32 = nullptr;
    float* z32 = nullptr;   // FP32 copy of the linearisation point (mixed precision)
    int64_t ndof = 0;
};
int64_t dg1_lin_flux_len(const DevParams& p);
// vertex-based slope limiter of the liquid species of a DG1 state (scratch: NL x n_cell doubles)
cudaError_t dg1_limit(const LaunchCtx& L, const DevParams& p, const Geo& g, double* z, double* scratch);
// per-node diagonal blocks of S J (dt-scaled rows) from a current linearisation at z
cudaError_t dg1_lin_blocks(const LaunchCtx& L, const DevParams& p, const Geo& g, const double* z, double dt, int relax,
                           const DG1Lin& lin, double* blk);
int64_t dg1_lin_sizes(const DevParams& p, int64_t* jn, int64_t* gam, int64_t* face);
cudaError_t dg1_linearize(const LaunchCtx& L, const DevParams& p, const Geo& g, const double* z, double t, double dt,
                          int relax, const DG1Lin& lin);
template <class S>
cudaError_t dg1_lin_apply(const LaunchCtx& L, const DevParams& p, const Geo& g, const S* z, const S* v,
                          double t, double dt, int relax, double sc_dt, S* out, const DG1Lin& lin);

// ------------------------------------------------------------------ batched instances
// One record per instance of a batch (device memory); the batched kernels launch once over the
// block ranges of all instances of one kind, and launch block b runs block map[b].y of instance
// map[b].x with the same device functions as the single-instance kernels (map: the schedule).
template <class S>
struct alignas(16) Job0 {          // DG0: transport factors, then the residual or the product
    DevParams p;
    Geo g;
    const S* z;
    const S* v;
    const double* zn;
    S* gb;
    S* gbd;
    S* out;
    double t, dt, sc_dt;
    int relax;
};
template <class S>
cudaError_t dg0_batch(const LaunchCtx& L, bool tradeoff, int mode, const Job0<S>* d_jobs, const int2* d_map,
                      int nblk, int bs);
// largest block size every batched DG0 product kernel of this chemistry and precision can launch with
int dg0_batch_max_block(bool tradeoff, bool f32);
// DG1 fused product: job records are opaque bytes of dg1_job_bytes(f32), filled on the host
size_t dg1_job_bytes(bool f32);
void dg1_fused_job(bool f32, const DevParams& p, const Geo& g, const void* z, const void* v, double t, double dt,
                   int relax, double sc_dt, void* out, void* job);
cudaError_t dg1_jvp_fused_batched(const LaunchCtx& L, bool f32, bool tradeoff, const void* d_jobs, const int2* d_map,
                                  int nblk);
// FP64 -> FP32 copies of several vectors in one launch (blocks of 256 x 4 elements)
struct ConvJob {
    const double* src;
    float* dst;
    int64_t n;
};
cudaError_t to_f32_batched(const LaunchCtx& L, const ConvJob* d_jobs, const int2* d_map, int nblk);
constexpr int CONV_BLOCK_ELEMS = 1024;
constexpr int FUSED_VOXELS = 32;   // voxels per block of the fused DG1 product
constexpr size_t JOB_SLOT = 4096;  // bytes of one job-record slot (every job record fits)

// ------------------------------------------------------------------ linear algebra (la.cu)
// Block-Jacobi: invert nblk blocks of nf x nf (row-major) in place; identity rows for absent
// fields are set by the builders.  Returns the count of singular blocks in *bad (device).
cudaError_t block_invert(const LaunchCtx& L, double* blk, int64_t nblk, int nf, float* blk32, int* bad);
template <class S>
cudaError_t block_apply(const LaunchCtx& L, const DevParams& p, const Geo& g, const void* blk,
                        const S* v, S* out);
template <class S>
cudaError_t mdot(const LaunchCtx& L, const S* V, int64_t ld, int64_t n, int k, const S* w,
                 double* partial, double* out, bool self = false);
template <class S>
cudaError_t maxpy_norm(const LaunchCtx& L, S* w, const S* V, int64_t ld, int64_t n, int k, const double* h,
                       double* partial, double* nrm2);
template <class S>
cudaError_t maxpy(const LaunchCtx& L, S* w, const S* V, int64_t ld, int64_t n, int k, const double* h,
                  double sign);
template <class S>
cudaError_t scale_copy(const LaunchCtx& L, S* dst, const S* src, int64_t n, const double* inv_norm_dev, double a);
template <class S>
cudaError_t neg_scaled(const LaunchCtx& L, const DevParams& p, const double* r, double dt, S* out);
cudaError_t scaled_norm2(const LaunchCtx& L, const DevParams& p, const double* r, double dt,
                         double* partial, double* out);
cudaError_t axpby(const LaunchCtx& L, double* y, double a, const double* x, double b, int64_t n);
cudaError_t to_f32(const LaunchCtx& L, float* dst, const double* src, int64_t n);
cudaError_t to_f64_add(const LaunchCtx& L, double* dst, const float* src, double a, int64_t n);
cudaError_t row_scales(const LaunchCtx& L, const DevParams& p, double dt, double* s);
cudaError_t fill_equilibrium(const LaunchCtx& L, const DevParams& p, const double* vals, double* z);
cudaError_t reduce_sum(const LaunchCtx& L, const double* x, int64_t n, double* partial, double* out);
cudaError_t cell_voltage(const LaunchCtx& L, const DevParams& p, const Geo& g, const double* z,
                         double* partial, double* out);
cudaError_t ledger(const LaunchCtx& L, const DevParams& p, const Geo& g, const double* z,
                   double* partial, double* out5);

// ------------------------------------------------------------------ potential multigrid (mg.cu)
cudaError_t mg_levels_alloc(std::vector<MGLevel>& lv, int nx, int ny, int nz, std::vector<void*>& allocs,
                            int64_t* bytes, DevArena* arena = nullptr);
cudaError_t mg_setup(const LaunchCtx& L, const DevParams& p, const Geo& g, const double* z, const double* gb,
                     double t, double dt, int relax, std::vector<MGLevel>& lv);
template <class S>
cudaError_t cpr_stage1(const LaunchCtx& L, const DevParams& p, const Geo& g, std::vector<MGLevel>& lv, int cycles,
                       const S* v, S* y);
// species coarse level: one two-field hierarchy per pair of liquid species (2k, 2k+1), level 0 from the
// transport factors gb and, for DG1, the node Jacobians jn (FP32 when jn_f32) at the linearisation point
cudaError_t mg_species_setup(const LaunchCtx& L, const DevParams& p, const Geo& g, const double* z, const double* gb,
                             const void* jn, bool jn_f32, double t, double dt, std::vector<MGLevel>* lv, int npairs);
// y += sum over the pairs of P V-cycle(P^T v) on the pair's species rows
template <class S>
cudaError_t mg_species_apply(const LaunchCtx& L, const DevParams& p, std::vector<MGLevel>* lv, int npairs, const S* v,
                             S* y);
template <class S>
cudaError_t saxpby(const LaunchCtx& L, S* y, double a, const S* x, double b, int64_t n);

constexpr int RED_BLOCKS = 1216;   // 8 x 152 SMs: fixed grid so that reductions are deterministic
constexpr int RED_THREADS = 256;
constexpr int MAXK = 32;           // GMRES restart + 1 upper bound for the fused dot kernels

}  // namespace dgls
