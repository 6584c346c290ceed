// Fused matrix-free DG1 Jacobian-vector product: J(z) v in one launch, reading z and v once and
// writing J v once (the 12 bytes per unknown of an FP32 product, 24 of an FP64 one).
//
// J v is the directional derivative of the DG1 residual (Eqs. 43-48 with the Tab. 4 system and
// the Tab. 3 sources) at z along v, evaluated with forward-mode dual numbers; nothing is cached
// between products, so the Krylov loop of the mixed-precision solver streams only its vectors.
//
// Mapping: one thread block per 32 consecutive voxels, one warp per DG1 node (8 warps), lane =
// voxel.  Every field of a node plane is contiguous in the node-major layout, so each warp load is
// one 128-byte (FP32) request.
//   phase 0  the block's nodal values of z and v go to shared memory;
//   phase 1  each thread evaluates, at its node, the transport factor g (Eqs. 2-3, 18) and the
//            node terms (storage, Eq. 50, and reaction sources), and g at the three face points
//            on its side of its three nodal lines;
//   phase 2  per direction, the volume term of the thread's line (both nodes of a line are in the
//            block) and the interior-penalty flux (Eq. 46) through the face point on its side, from
//            its own traces and the neighbour voxel's: the x-neighbour of an inner lane is read
//            from shared memory, other neighbours from global memory (in practice from L2: the
//            blocks that own them, mostly on other SMs, read the same values), all twenty (z, v)
//            pairs of a face loaded together;
//   phase 3  each node adds its own face flux (trace weight ALPHA) and its line partner's (BETA)
//            from shared memory and stores its row-scaled outputs.
// Each interior face point is evaluated by the voxels on both of its sides; from the same inputs
// the two results are exact negatives of each other (see phase 2), and the inputs agree bit for bit
// except for the neighbour's face-point transport factor, which a side whose neighbour is in
// another block recomputes.
//
// The kernel always runs from a table of job records (one per instance: parameters, geometry,
// buffers, per-call constants) and a block map: a batch of many instances and a single instance
// (a one-job table) use the same compiled kernel, so an instance's product is bitwise the same
// alone and in a batch.
#include <cstring>

#include "dg1_shared.cuh"

namespace dgls {

namespace {
constexpr int FT = 32;   // voxels per block

// per-call constants in the arithmetic type of the product (FP32 products stay on the FP32 pipe)
template <class S>
struct FusedK {
    S wf, vol, pen, gq2;            // face weight (h/2)^2, volume weight 3h/8, penalty / h, sqrt(3) / (2h)
    S D0[6], km[6], Kd[6], Km[6];   // species row: D0 and z F/(RT) D0 (zero while relaxing); Phi^L row
    S kSv, kS;                      // Phi^S: 2 kappa_s vol in the volume, kappa_s at faces
    S aLi, aL;                      // anode: k_Ano on the Li+ row (zero while relaxing), F k_Ano on Phi^L
    S rs[DG_MAXF];                  // row scales of the outputs (Newton rows) or 1
    S M, Mdt, Msdt[2];              // node volume h^3/8, M/dt, M rho_s/(M_s dt) of the two solids
    S tH;                           // T_H(t) of Eq. 56 (the smoothed reactions)
    int charged;                    // bit m: species m carries charge
};

// line index q of node n in direction d (the node's two coordinates across d)
__device__ __forceinline__ int line_of(int d, int n) {
    const int a = n & 1, b = (n >> 1) & 1, c = (n >> 2) & 1;
    return d == 0 ? b + 2 * c : d == 1 ? a + 2 * c : a + 2 * b;
}

template <class Chem>
__host__ __device__ constexpr bool struct_field(int f) {
    return (f >= Chem::NL && f < Chem::NL + Chem::NS) || f == Chem::PHIS;
}

// Tangent of the node terms of one DG1 node (mass M = h^3/8): storage of Eq. 50 (or the d_t Phi
// terms of the relaxation of Sec. 2.8) minus the reaction sources of structure points (Tab. 4);
// the previous time level enters the node terms as constants only, so it drops out.
template <class Chem, class S>
__device__ __forceinline__ void node_tangent(const DevParams& p, const FusedK<S>& K, int ph, const Dual<S>* c,
                                             const Dual<S>* es, Dual<S> phiL, Dual<S> phiS, int relax, S* out) {
    typedef Dual<S> T;
    constexpr int NL = Chem::NL, NS = Chem::NS, PHIL = Chem::PHIL, PHIS = Chem::PHIS;
    const bool st = ph == 1;
    const T epsL = liquid_fraction<Chem, T>(p, ph, es);
#pragma unroll
    for (int m = 0; m < NL; ++m) out[m] = (relax ? c[m].d : (epsL * c[m]).d) * K.Mdt;
#pragma unroll
    for (int q = 0; q < NS; ++q) out[NL + q] = st ? es[q].d * K.Msdt[q] : S(0);
    out[PHIL] = relax ? phiL.d * K.Mdt : S(0);
    out[PHIS] = relax && st ? phiS.d * K.Mdt : S(0);
    if (st) {
        T Sv[NL], Ss[2], qL, qS;
        sources<Chem, T>(p, c, es, phiL, phiS, K.tH, Sv, Ss, qL, qS);
        if (!relax) {
#pragma unroll
            for (int m = 0; m < NL; ++m) out[m] -= Sv[m].d * K.M;
#pragma unroll
            for (int q = 0; q < NS; ++q) out[NL + q] -= Ss[q].d * K.M;
        }
        out[PHIL] -= qL.d * K.M;
        out[PHIS] -= qS.d * K.M;
    }
}

template <class Chem, class S>
__host__ __device__ constexpr size_t fused_smem() {
    return (size_t)(2 * Chem::NF * 8 * FT + 2 * 32 * FT + 8 * 3 * (Chem::NL + 2) * FT) * sizeof(S) + 2 * FT * sizeof(int);
}

// one instance of a batched product
template <class S>
struct alignas(16) Job1 {
    DevParams p;
    Geo g;
    FusedK<S> K;
    const S* z;
    const S* v;
    S* out;
    int relax;
};
static_assert(FT == FUSED_VOXELS, "block width");
}  // namespace

// The product over one block of 32 voxels (block index `blk` of the instance); the calling kernel
// provides the dynamic shared memory (fused_smem bytes) and 256 threads.
template <class Chem, class S>
__device__ __forceinline__ void jvp1_block(const DevParams& p, const Geo& g, const S* __restrict__ z,
                                           const S* __restrict__ v, const FusedK<S>& K, int relax,
                                           S* __restrict__ out, int blk, unsigned char* smem_raw) {
    typedef Dual<S> T;
    constexpr int NL = Chem::NL, NS = Chem::NS, NF = Chem::NF, PHIL = Chem::PHIL, PHIS = Chem::PHIS;
    constexpr int NE = NL + 2;   // transport equations: the species, Phi^L, Phi^S
    typedef typename std::conditional<std::is_same<S, float>::value, float2, double2>::type S2;
    S2* sZV = reinterpret_cast<S2*>(smem_raw);   // [NF][8][FT] (z, v) pairs: one shared load per value and tangent
    S* sG = reinterpret_cast<S*>(sZV + NF * 8 * FT);   // [32 slots][FT] transport factors (value)
    S* sGd = sG + 32 * FT;                    // [32 slots][FT] (tangent)
    S* sF = sGd + 32 * FT;                    // [8 nodes][3 dirs][NE][FT] near-face flux tangents, signed and weighted
    int* sPh = reinterpret_cast<int*>(sF + 8 * 3 * NE * FT);
    int* sSi = sPh + FT;

    const int n = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blk * FT + lane;
    const bool active = c < p.n_cell;
    const S al = S(ALPHA), be = S(BETA);

    // ---- phase 0: the block's nodal values
    int ph = 0, si = -1;
    if (active) {
        ph = g.phase[c];
        si = g.cmap[c];
    }
    if (n == 0) {
        sPh[lane] = ph;
        sSi[lane] = si;
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        S zz = S(0), vv = S(0);
        if (active && (!struct_field<Chem>(f) || ph == 1)) {
            const int64_t o = p.off[f] + (int64_t)n * p.flen[f] + (struct_field<Chem>(f) ? si : c);
            zz = z[o];
            vv = v[o];
        }
        S2 w;
        w.x = zz;
        w.y = vv;
        sZV[(f * 8 + n) * FT + lane] = w;
    }
    __syncthreads();
    auto zv = [&](int f, int node, int l) -> T {
        const S2 w = sZV[(f * 8 + node) * FT + l];
        return mkd(w.x, w.y);
    };

    // ---- phase 1: transport factors at the node and its three face points; node terms
    S acc[NF];
    {
        T cn[NL], es[2];
#pragma unroll
        for (int m = 0; m < NL; ++m) cn[m] = zv(m, n, lane);
        es[0] = es[1] = Make<T>::c(0.0);
        if (NS == 2 && ph == 1) {
            es[0] = zv(NL, n, lane);
            es[1] = zv(NL + 1, n, lane);
        }
        {
            const T gg = transport_factor<Chem, T>(p, liquid_fraction<Chem, T>(p, ph, es), cn);
            sG[n * FT + lane] = gg.v;
            sGd[n * FT + lane] = gg.d;
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int pn = n ^ (1 << d);
            const int side = (n >> d) & 1 ? 1 : -1;
            T ct[NL], et[2];
#pragma unroll
            for (int m = 0; m < NL; ++m) ct[m] = cn[m] * al + zv(m, pn, lane) * be;
            et[0] = et[1] = Make<T>::c(0.0);
            if (NS == 2 && ph == 1) {
                et[0] = es[0] * al + zv(NL, pn, lane) * be;
                et[1] = es[1] * al + zv(NL + 1, pn, lane) * be;
            }
            const T gg = transport_factor<Chem, T>(p, liquid_fraction<Chem, T>(p, ph, et), ct);
            const int slot = face_slot(d, side, line_of(d, n));
            sG[slot * FT + lane] = gg.v;
            sGd[slot * FT + lane] = gg.d;
        }
        // storage and sources of this node
        const T phiL = zv(PHIL, n, lane);
        const T phiS = ph == 1 ? zv(PHIS, n, lane) : Make<T>::c(0.0);
        node_tangent<Chem, S>(p, K, ph, cn, es, phiL, phiS, relax, acc);
    }
    __syncthreads();

    // ---- phase 2: per direction, the line's volume term and the flux through this node's face point
    int ci = 0, cj = 0, ck = 0;
    if (active) cell_ijk(p, c, ci, cj, ck);
#pragma unroll 1   // one copy of the direction body: the kernel is large, and instruction fetch stalled it
    for (int d = 0; d < 3; ++d) {
        const int pn = n ^ (1 << d);
        const int mc = (n >> d) & 1;         // this node's coordinate along d (1: next to the +d face)
        const int n0 = mc ? pn : n, n1 = mc ? n : pn;
        // volume term of the line (n0, n1): n1 gets +fl, n0 gets -fl
        {
            const S sgn = mc ? S(1) : S(-1);
            const T gN0 = mkd(sG[n0 * FT + lane], sGd[n0 * FT + lane]);
            const T gN1 = mkd(sG[n1 * FT + lane], sGd[n1 * FT + lane]);
            const T gsum = gN0 + gN1;
            const T dPhi = zv(PHIL, n1, lane) - zv(PHIL, n0, lane);
            S accL = S(0);
#pragma unroll
            for (int m = 0; m < NL; ++m) {
                const T C0 = zv(m, n0, lane), C1 = zv(m, n1, lane);
                const T gdc = gsum * (C1 - C0);
                S fl = (gdc * K.D0[m]).d;
                if ((K.charged >> m) & 1) {
                    const T mdp = (gN0 * C0 + gN1 * C1) * dPhi;
                    fl += (mdp * K.km[m]).d;
                    accL += (gdc * K.Kd[m] + mdp * K.Km[m]).d;
                }
                acc[m] += sgn * K.vol * fl;
            }
            acc[PHIL] += sgn * K.vol * accL;
            if (ph == 1) acc[PHIS] += sgn * K.kSv * (zv(PHIS, n1, lane).d - zv(PHIS, n0, lane).d);
        }
        // flux through the face point on this node's side of the line
        S Fe[NE];
#pragma unroll
        for (int e = 0; e < NE; ++e) Fe[e] = S(0);
        const int coord = d == 0 ? ci : d == 1 ? cj : ck;
        const int ext = d == 0 ? p.nx : d == 1 ? p.ny : p.nz;
        const int stride = d == 0 ? 1 : d == 1 ? p.nx : p.nx * p.ny;
        const bool hasQ = active && (mc ? coord + 1 < ext : coord > 0);
        if (hasQ) {
            const int qc = c + (mc ? stride : -stride);
            const int ql = lane + (mc ? 1 : -1);
            const bool local = d == 0 && ql >= 0 && ql < FT;
            const int qph = local ? sPh[ql] : g.phase[qc];
            const int qsi = local ? sSi[ql] : g.cmap[qc];
            // the neighbour's values at its near node (pn) and its far node (n), all loads issued
            // together so that one L2 round trip covers them
            T qN[NF], qF[NF];
            if (local) {
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    qN[f] = zv(f, pn, ql);
                    qF[f] = zv(f, n, ql);
                }
            } else {
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    if (struct_field<Chem>(f) && qph != 1) {
                        qN[f] = qF[f] = Make<T>::c(0.0);
                    } else {
                        const int64_t b = p.off[f] + (struct_field<Chem>(f) ? qsi : qc);
                        const int64_t o0 = b + (int64_t)pn * p.flen[f], o1 = b + (int64_t)n * p.flen[f];
                        qN[f] = mkd(z[o0], v[o0]);
                        qF[f] = mkd(z[o1], v[o1]);
                    }
                }
            }
            const int q = line_of(d, n);
            const int slotP = face_slot(d, mc ? 1 : -1, q);
            const T gP = mkd(sG[slotP * FT + lane], sGd[slotP * FT + lane]);
            T gQ;
            if (local) {
                const int slotQ = face_slot(d, mc ? -1 : 1, q);
                gQ = mkd(sG[slotQ * FT + ql], sGd[slotQ * FT + ql]);
            } else {
                T ct[NL], et[2];
#pragma unroll
                for (int m = 0; m < NL; ++m) ct[m] = qN[m] * al + qF[m] * be;
                et[0] = et[1] = Make<T>::c(0.0);
                if (NS == 2 && qph == 1) {
                    et[0] = qN[NL] * al + qF[NL] * be;
                    et[1] = qN[NL + 1] * al + qF[NL + 1] * be;
                }
                gQ = transport_factor<Chem, T>(p, liquid_fraction<Chem, T>(p, qph, et), ct);
            }
            // Everything below is taken from this voxel's side: the bracket with the own trace first
            // is the left-minus-right bracket times sgn = +1 (this voxel left of the face) or -1, and
            // the flux is linear in the brackets, so the flux from this side is sgn times the face
            // flux, exactly (negation is exact and the harmonic means are symmetric to the last
            // bit); the stored value (flux from this side) x wf is then +f for the left voxel and -f
            // for the right one, with no selects on the side.
            const T Hg = harm(gP, gQ);
            auto bracket = [&](T own_n, T own_f, T nb_n, T nb_f, T& t_own, T& t_nb) -> T {
                t_own = own_n * al + own_f * be;
                t_nb = nb_n * al + nb_f * be;
                const T dn = ((own_n - own_f) + (nb_f - nb_n)) * K.gq2;
                return (t_own - t_nb) * K.pen - dn;
            };
            T tPo, tPn;
            const T bL = bracket(zv(PHIL, n, lane), zv(PHIL, pn, lane), qN[PHIL], qF[PHIL], tPo, tPn);
            S fL = S(0);
#pragma unroll
            for (int m = 0; m < NL; ++m) {
                T to, tn;
                const T b = bracket(zv(m, n, lane), zv(m, pn, lane), qN[m], qF[m], to, tn);
                const T dterm = b * Hg;
                S f = (dterm * K.D0[m]).d;
                if ((K.charged >> m) & 1) {
                    const T mterm = bL * harm(gP * to, gQ * tn);
                    f += (mterm * K.km[m]).d;
                    fL += (dterm * K.Kd[m] + mterm * K.Km[m]).d;
                }
                Fe[m] = f;
            }
            Fe[NL] = fL;
            if (ph == 1 && qph == 1) {
                const S jn = zv(PHIS, n, lane).d, jf = zv(PHIS, pn, lane).d;
                const S qn = qN[PHIS].d, qf = qF[PHIS].d;
                const S to = jn * al + jf * be, tn = qn * al + qf * be;
                const S dn = ((jn - jf) + (qf - qn)) * K.gq2;
                Fe[NL + 1] = ((to - tn) * K.pen - dn) * K.kS;
            }
        } else if (active && d == 0 && mc && ci == p.nx - 1) {
            // anode face (Eqs. 26-27): exchange rate at the face trace of c_Li and Phi^L
            const T cLi = zv(0, n, lane) * al + zv(0, pn, lane) * be;
            const T phL = zv(PHIL, n, lane) * al + zv(PHIL, pn, lane) * be;
            const S rA = anode_rate<T>(p, cLi, phL).d;
            Fe[0] = rA * K.aLi;
            Fe[NL] = rA * K.aL;
        }
        // flux from this side x the face weight: +f for the left voxel of the face, -f for the right
        // one (the anode face has its voxel on the left)
#pragma unroll
        for (int e = 0; e < NE; ++e) sF[((n * 3 + d) * NE + e) * FT + lane] = Fe[e] * K.wf;
    }
    __syncthreads();

    // ---- phase 3: own face flux (near node, ALPHA) and the partner's (far node, BETA); store
    if (!active) return;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int pn = n ^ (1 << d);
#pragma unroll
        for (int e = 0; e < NE; ++e) {
            const int f = e < NL ? e : e == NL ? PHIL : PHIS;
            acc[f] += al * sF[((n * 3 + d) * NE + e) * FT + lane] + be * sF[((pn * 3 + d) * NE + e) * FT + lane];
        }
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        if (struct_field<Chem>(f) && ph != 1) continue;
        const int64_t o = p.off[f] + (int64_t)n * p.flen[f] + (struct_field<Chem>(f) ? si : c);
        out[o] = acc[f] * K.rs[f];
    }
}

// Batched product: launch block b runs block map[b].y of instance map[b].x, whose job record is
// staged in shared memory behind the product's own arrays.
template <class Chem, class S>
__global__ void __launch_bounds__(256, sizeof(S) == 4 ? 3 : 1) k_jvp1_batched(const Job1<S>* __restrict__ jobs,
                                                                             const int2* __restrict__ map) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr size_t off = (fused_smem<Chem, S>() + 15) / 16 * 16;
    Job1<S>* sj = reinterpret_cast<Job1<S>*>(smem_raw + off);
    {
        const int4* src = reinterpret_cast<const int4*>(jobs + map[blockIdx.x].x);
        int4* dst = reinterpret_cast<int4*>(sj);
        for (int w = threadIdx.x; w < (int)(sizeof(Job1<S>) / 16); w += blockDim.x) dst[w] = src[w];
    }
    __syncthreads();
    jvp1_block<Chem, S>(sj->p, sj->g, sj->z, sj->v, sj->K, sj->relax, sj->out, map[blockIdx.x].y, smem_raw);
}

template <class S>
static void fill_K(const DevParams& p, int nl, int nf, double t, double dt, int relax, double sc_dt, FusedK<S>& K) {
    const double h = p.h;
    K.wf = S(0.25 * h * h);
    K.vol = S(3.0 * h / 8.0);
    K.pen = S(p.penalty / h);
    K.gq2 = S(0.5 * 1.7320508075688772935 / h);
    K.charged = 0;
    for (int m = 0; m < 6; ++m) {
        const bool on = m < nl;
        K.D0[m] = S(on && !relax ? p.D0[m] : 0.0);
        K.km[m] = S(on && !relax ? p.kappa_m[m] : 0.0);
        K.Kd[m] = S(on ? p.Kd[m] : 0.0);
        K.Km[m] = S(on ? p.Km[m] : 0.0);
        if (on && p.zc[m] != 0.0) K.charged |= 1 << m;
    }
    K.kSv = S(2.0 * p.kappa_s * 3.0 * h / 8.0);
    K.kS = S(p.kappa_s);
    K.aLi = S(relax ? 0.0 : p.kAno);
    K.aL = S(p.F * p.kAno);
    for (int f = 0; f < DG_MAXF; ++f) K.rs[f] = S(f < nf && sc_dt > 0.0 ? sc_dt * p.rscale[f] : 1.0);
    const double M = p.V / 8.0;
    K.M = S(M);
    K.Mdt = S(M / dt);
    K.Msdt[0] = S(M * p.rhoM[0] / dt);
    K.Msdt[1] = S(M * p.rhoM[1] / dt);
    K.tH = S(smooth_step(t));
}

static_assert(sizeof(Job1<double>) <= JOB_SLOT && sizeof(Job1<float>) <= JOB_SLOT, "job record slot");
size_t dg1_job_bytes(bool f32) { return f32 ? sizeof(Job1<float>) : sizeof(Job1<double>); }

template <class S>
static void fill_job(const DevParams& p, const Geo& g, const void* z, const void* v, double t, double dt, int relax,
                     double sc_dt, void* out, void* job) {
    Job1<S> J;
    std::memset(&J, 0, sizeof(J));
    J.p = p;
    J.g = g;
    fill_K<S>(p, p.nl, p.nf, t, dt, relax, sc_dt, J.K);
    J.z = (const S*)z;
    J.v = (const S*)v;
    J.out = (S*)out;
    J.relax = relax;
    std::memcpy(job, &J, sizeof(J));
}

void dg1_fused_job(bool f32, const DevParams& p, const Geo& g, const void* z, const void* v, double t, double dt,
                   int relax, double sc_dt, void* out, void* job) {
    if (f32) fill_job<float>(p, g, z, v, t, dt, relax, sc_dt, out, job);
    else fill_job<double>(p, g, z, v, t, dt, relax, sc_dt, out, job);
}

template <class Chem, class S>
static cudaError_t batched_impl(const LaunchCtx& L, const void* d_jobs, const int2* d_map, int nblk) {
    const size_t smem = (fused_smem<Chem, S>() + 15) / 16 * 16 + sizeof(Job1<S>);
    cudaError_t e = cudaFuncSetAttribute(k_jvp1_batched<Chem, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_jvp1_batched<Chem, S><<<nblk, 8 * FT, smem, L.st>>>((const Job1<S>*)d_jobs, d_map);
    *L.counter += 1;
    return cudaGetLastError();
}

cudaError_t dg1_jvp_fused_batched(const LaunchCtx& L, bool f32, bool tradeoff, const void* d_jobs, const int2* d_map,
                                  int nblk) {
    if (nblk <= 0) return cudaSuccess;
    if (f32) return tradeoff ? batched_impl<ChemTO, float>(L, d_jobs, d_map, nblk)
                             : batched_impl<ChemR3, float>(L, d_jobs, d_map, nblk);
    return tradeoff ? batched_impl<ChemTO, double>(L, d_jobs, d_map, nblk)
                    : batched_impl<ChemR3, double>(L, d_jobs, d_map, nblk);
}

}  // namespace dgls
