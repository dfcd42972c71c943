// Device bodies of the float64 kernels of a step (sdc.cu): the implicit
// right-hand side F_I, the SDC node updates with their implicit solve
// (Sec. 4.2, Sec. 4.4), the node broadcast, the MLSDC transfers (Sec. 4.3,
// Algorithm 1) and the device copy the persistent ensemble kernel runs in
// place of cudaMemcpy2DAsync.  Each takes its block index, threads, barrier
// and shared memory from a Blk (vblock.cuh): sdc.cu's kernels pass the
// hardware values, persistent.cu runs them for virtual blocks.  Pointer
// arguments carry no __restrict__ here: inside the persistent kernel a buffer
// read by one phase is written by another.
#pragma once

#include "internal.h"
#include "sdc_internal.h"

namespace mlsdc {

// dt-scaled rows 1..M of Q, Q_E, Q_I (the sweep-constant node update)
struct SweepMats {
    double q[kMaxNodes][kMaxNodes], qe[kMaxNodes][kMaxNodes], qi[kMaxNodes][kMaxNodes];
};

// shared memory of a node-update block: the three fields' right-hand sides
constexpr size_t kNodeSmem = 3 * kNodeCoefs * sizeof(double2);

__device__ __forceinline__ void b_implicit_rhs(const Blk& bk, const double2* x, double2* F, const int* ndeg, int nc, Phys ph, size_t ms_x, size_t ms_f) {
    pdl_wait();
    pdl_launch();
    x += bk.idx.y * ms_x;
    F += bk.idx.y * ms_f;
    for (int c = bk.idx.x * bk.nt + bk.t; c < nc; c += bk.dim.x * bk.nt) {
        const double n = ndeg[c];
        const double L = -n * (n + 1.0) * ph.inv_a2;
        double2 fp, fz, fd;
        implicit_rhs_coef(L, ph, x[c], x[nc + c], x[2 * nc + c], fp, fz, fd);
        F[c] = fp;
        F[nc + c] = fz;
        F[2 * nc + c] = fd;
    }
}

__device__ __forceinline__ void b_sweep_node(const Blk& bk, double2* Th, const double2* FIo, const double2* FEo, double2* FIn, double2* FEn, const double2* tau, const int* ndeg, const double2* recips, int nc, const NodeRow& row, Phys ph, size_t ms) {
    double2(*sb)[kNodeCoefs] = reinterpret_cast<double2(*)[kNodeCoefs]>(bk.smem);
    pdl_wait();
    pdl_launch();
    const size_t mo = bk.idx.y * ms;
    Th += mo;
    FIo += mo;
    FEo += mo;
    FIn += mo;
    FEn += mo;
    if (tau) tau += mo;
    const size_t node = (size_t)3 * nc;
    const int m = row.m;
    const int f = bk.t / kNodeCoefs, cl = bk.t - f * kNodeCoefs;
    const int c = bk.idx.x * kNodeCoefs + cl;
    const bool live = c < nc;
    const size_t o = (size_t)f * nc + c;
    // the degree and the solve reciprocals (constant tables): loaded ahead, their latency under the sums
    int nd = 0;
    double2 rc = make_double2(0.0, 0.0);
    if (live) {
        nd = ndeg[c];
        rc = recips[nd];
    }
    if (live) sb[f][cl] = node_rhs(Th, FIo, FEo, FIn, FEn, tau, node, o, row);
    bk.sync();
    if (!live) return;
    const double n = nd;
    const double L = -n * (n + 1.0) * ph.inv_a2;
    double2 th, fi;  // each thread only its own field (warp-uniform f)
    node_solve_field(f, L, row.qimm, ph, rc, sb[0][cl], sb[1][cl], sb[2][cl], th, fi);
    const size_t om = (m + 1) * node + o;
    Th[om] = th;
    FIn[om] = fi;
    if (m == 0) {
        FIn[o] = FIo[o];
        FEn[o] = FEo[o];
    }
}

template <int MM>
__device__ __forceinline__ void b_sweep_node0(const Blk& bk, double2* Th, const double2* FIo, const double2* FEo, double2* FIn, double2* FEn, const double2* tau, double2* S, const int* ndeg, const double2* recips, int nc, const SweepMats& sm, Phys ph, size_t ms, size_t ms_s) {
    double2(*sb)[kNodeCoefs] = reinterpret_cast<double2(*)[kNodeCoefs]>(bk.smem);
    pdl_wait();
    pdl_launch();
    const size_t mo = bk.idx.y * ms;
    Th += mo;
    FIo += mo;
    FEo += mo;
    FIn += mo;
    FEn += mo;
    if (tau) tau += mo;
    S += bk.idx.y * ms_s;
    const size_t node = (size_t)3 * nc;
    const int f = bk.t / kNodeCoefs, cl = bk.t - f * kNodeCoefs;
    const int c = bk.idx.x * kNodeCoefs + cl;
    const bool live = c < nc;
    const size_t o = (size_t)f * nc + c;
    // the degree and the solve reciprocals (constant tables): loaded ahead, their latency under the sums
    int nd = 0;
    double2 rc = make_double2(0.0, 0.0);
    if (live) {
        nd = ndeg[c];
        rc = recips[nd];
    }
    if (live) {
        double2 acc[MM + 1];
        const double2 t0 = Th[o];
#pragma unroll
        for (int r = 1; r <= MM; ++r) acc[r] = tau ? make_double2(t0.x + tau[r * node + o].x, t0.y + tau[r * node + o].y)
                                                   : t0;
#pragma unroll
        for (int j = 0; j <= MM; ++j) {
            const double2 fi = FIo[j * node + o], fe = FEo[j * node + o];
            const double2 s = make_double2(fi.x + fe.x, fi.y + fe.y);
#pragma unroll
            for (int r = 1; r <= MM; ++r) {
                acc[r] = cax(acc[r], sm.q[r][j], s);
                if (j >= 1 && j < r) {
                    acc[r] = cax(acc[r], -sm.qe[r][j], fe);
                    acc[r] = cax(acc[r], -sm.qi[r][j], fi);
                } else if (j == r) {
                    acc[r] = cax(acc[r], -sm.qi[r][r], fi);
                }
            }
        }
#pragma unroll
        for (int r = 2; r <= MM; ++r) S[(r - 2) * node + o] = acc[r];
        sb[f][cl] = acc[1];
    }
    bk.sync();
    if (!live) return;
    const double n = nd;
    const double L = -n * (n + 1.0) * ph.inv_a2;
    double2 th, fi;
    node_solve_field(f, L, sm.qi[1][1], ph, rc, sb[0][cl], sb[1][cl], sb[2][cl], th, fi);
    Th[node + o] = th;
    FIn[node + o] = fi;
    FIn[o] = FIo[o];
    FEn[o] = FEo[o];
}

__device__ __forceinline__ void b_sweep_node_s(const Blk& bk, double2* Th, double2* FIn, const double2* FEn, const double2* S, const int* ndeg, const double2* recips, int nc, const NodeRow& row, Phys ph, size_t ms, size_t ms_s) {
    double2(*sb)[kNodeCoefs] = reinterpret_cast<double2(*)[kNodeCoefs]>(bk.smem);
    pdl_wait();
    pdl_launch();
    const size_t mo = bk.idx.y * ms;
    Th += mo;
    FIn += mo;
    FEn += mo;
    S += bk.idx.y * ms_s;
    const size_t node = (size_t)3 * nc;
    const int m = row.m;
    const int f = bk.t / kNodeCoefs, cl = bk.t - f * kNodeCoefs;
    const int c = bk.idx.x * kNodeCoefs + cl;
    const bool live = c < nc;
    const size_t o = (size_t)f * nc + c;
    // the degree and the solve reciprocals (constant tables): loaded ahead, their latency under the sums
    int nd = 0;
    double2 rc = make_double2(0.0, 0.0);
    if (live) {
        nd = ndeg[c];
        rc = recips[nd];
    }
    if (live) {
        double2 acc = S[(m - 1) * node + o];
        for (int j = 1; j <= m; ++j) {
            acc = cax(acc, row.qe[j], FEn[j * node + o]);
            acc = cax(acc, row.qi[j], FIn[j * node + o]);
        }
        sb[f][cl] = acc;
    }
    bk.sync();
    if (!live) return;
    const double n = nd;
    const double L = -n * (n + 1.0) * ph.inv_a2;
    double2 th, fi;
    node_solve_field(f, L, row.qimm, ph, rc, sb[0][cl], sb[1][cl], sb[2][cl], th, fi);
    const size_t om = (m + 1) * node + o;
    Th[om] = th;
    FIn[om] = fi;
}

__device__ __forceinline__ void b_broadcast(const Blk& bk, const double2* src, double2* dst, int n3, int count, size_t ms_src, size_t ms_dst) {
    pdl_wait();
    pdl_launch();
    src += bk.idx.y * ms_src;
    dst += bk.idx.y * ms_dst;
    for (int c = bk.idx.x * bk.nt + bk.t; c < n3; c += bk.dim.x * bk.nt) {
        const double2 v = src[c];
        for (int k = 0; k < count; ++k) dst[(size_t)k * n3 + c] = v;
    }
}

__device__ __forceinline__ void b_restrict(const Blk& bk, const double2* Tf, double2* Tc, const int* c2f, int ncf, int ncc, int nf_nodes, int i0, int i1, const TransferMat& Pcf, size_t msf, size_t msc) {
    pdl_wait();
    pdl_launch();
    Tf += bk.idx.y * msf;
    Tc += bk.idx.y * msc;
    const int nc3 = 3 * ncc;
    const int total = (i1 - i0) * nc3;
    for (int t = bk.idx.x * bk.nt + bk.t; t < total; t += bk.dim.x * bk.nt) {
        const int i = i0 + t / nc3, r = t % nc3;
        const int f = r / ncc, k = r - f * ncc;
        const size_t of = (size_t)f * ncf + c2f[k];
        double2 acc{0.0, 0.0};
        for (int j = 0; j < nf_nodes; ++j) acc = cax(acc, Pcf.a[i * nf_nodes + j], Tf[(size_t)j * 3 * ncf + of]);
        Tc[(size_t)i * nc3 + r] = acc;
    }
}

__device__ __forceinline__ void b_fas_tau(const Blk& bk, const double2* Tf, const double2* FIf, const double2* FEf, const double2* Tc, const double2* FIc, const double2* FEc, double2* tau, double2* Ts, double2* FIs, double2* FEs, const double2* tauf, const int* c2f, int ncf, int ncc, const FasFwd& A, size_t msf, size_t msc) {
    pdl_wait();
    pdl_launch();
    const size_t of_m = bk.idx.y * msf, oc_m = bk.idx.y * msc;
    Tf += of_m;
    FIf += of_m;
    FEf += of_m;
    if (tauf) tauf += of_m;
    Tc += oc_m;
    FIc += oc_m;
    FEc += oc_m;
    tau += oc_m;
    Ts += oc_m;
    FIs += oc_m;
    FEs += oc_m;
    const int nc3 = 3 * ncc;
    const size_t nf3 = (size_t)3 * ncf;
    const int total = A.ncn * nc3;
    for (int t = bk.idx.x * bk.nt + bk.t; t < total; t += bk.dim.x * bk.nt) {
        const int i = t / nc3, r = t - i * nc3;
        const int f = r / ncc, k = r - f * ncc;
        const size_t of = (size_t)f * ncf + c2f[k];
        const size_t oc = (size_t)i * nc3 + r;
        const double2 tc = Tc[oc];
        Ts[oc] = tc;
        FIs[oc] = FIc[oc];
        FEs[oc] = FEc[oc];
        double2 acc = tc;
        for (int j = 0; j < A.nfn; ++j) {
            const size_t oj = (size_t)j * nf3 + of;
            const double2 sf = make_double2(FIf[oj].x + FEf[oj].x, FIf[oj].y + FEf[oj].y);
            acc = cax(acc, -A.Pcf[i * A.nfn + j], Tf[oj]);
            acc = cax(acc, A.dPQf[i * A.nfn + j], sf);
        }
        for (int l = 0; l < A.ncn; ++l) {
            const size_t ol = (size_t)l * nc3 + r;
            const double2 sc = make_double2(FIc[ol].x + FEc[ol].x, FIc[ol].y + FEc[ol].y);
            acc = cax(acc, -A.dQc[i * A.ncn + l], sc);
        }
        if (tauf)  // + R tau_f on a level below the finest (Eq. tau_term_level_l+1)
            for (int j = 0; j < A.nfn; ++j) acc = cax(acc, A.Pcf[i * A.nfn + j], tauf[(size_t)j * nf3 + of]);
        tau[oc] = acc;
    }
}

__device__ __forceinline__ void b_interp(const Blk& bk, double2* Tf, double2* FIf, double2* FEf, const double2* Tc, const double2* FIc, const double2* FEc, const double2* Ts, const double2* FIs, const double2* FEs, const int* c2f, int ncf, int ncc, int nfn, int ncn, const TransferMat& Pfc, size_t msf, size_t msc) {
    pdl_wait();
    pdl_launch();
    const size_t of_m = bk.idx.y * msf, oc_m = bk.idx.y * msc;
    Tf += of_m;
    FIf += of_m;
    FEf += of_m;
    Tc += oc_m;
    FIc += oc_m;
    FEc += oc_m;
    Ts += oc_m;
    FIs += oc_m;
    FEs += oc_m;
    const int nc3 = 3 * ncc;
    const size_t nf3 = (size_t)3 * ncf;
    const int total = (nfn - 1) * nc3;
    for (int t = bk.idx.x * bk.nt + bk.t; t < total; t += bk.dim.x * bk.nt) {
        const int m = 1 + t / nc3, r = t % nc3;
        const int f = r / ncc, k = r - f * ncc;
        const size_t of = (size_t)f * ncf + c2f[k];
        double2 aT{0, 0}, aI{0, 0}, aE{0, 0};
        for (int i = 0; i < ncn; ++i) {
            const double w = Pfc.a[m * ncn + i];
            if (w == 0.0) continue;
            const size_t oc = (size_t)i * nc3 + r;
            aT = cax(aT, w, make_double2(Tc[oc].x - Ts[oc].x, Tc[oc].y - Ts[oc].y));
            aI = cax(aI, w, make_double2(FIc[oc].x - FIs[oc].x, FIc[oc].y - FIs[oc].y));
            aE = cax(aE, w, make_double2(FEc[oc].x - FEs[oc].x, FEc[oc].y - FEs[oc].y));
        }
        const size_t o = (size_t)m * nf3 + of;
        Tf[o] = make_double2(Tf[o].x + aT.x, Tf[o].y + aT.y);
        FIf[o] = make_double2(FIf[o].x + aI.x, FIf[o].y + aI.y);
        FEf[o] = make_double2(FEf[o].x + aE.x, FEf[o].y + aE.y);
    }
}

__device__ __forceinline__ void b_pad_add(const Blk& bk, double2* Xf, const double2* Xc, const double2* X0, const int* c2f, int ncf, int ncc, size_t msf, size_t msc) {
    Xf += bk.idx.y * msf;
    Xc += bk.idx.y * msc;
    for (int t = bk.idx.x * bk.nt + bk.t; t < 3 * ncc; t += bk.dim.x * bk.nt) {
        const int f = t / ncc, k = t - f * ncc;
        const size_t o = (size_t)f * ncf + c2f[k];
        Xf[o] = make_double2(Xf[o].x + (Xc[t].x - X0[t].x), Xf[o].y + (Xc[t].y - X0[t].y));
    }
}

// `height` rows of `width` bytes (a multiple of 16, 16-byte aligned) from src
// (row pitch spitch bytes) to dst (pitch dpitch), one 16-byte word per thread
// and step: the step's copies inside the persistent ensemble kernel.
__device__ __forceinline__ void b_copy2d(const Blk& bk, unsigned char* dst, size_t dpitch, const unsigned char* src,
                                         size_t spitch, size_t width, int height) {
    const size_t wpr = width / 16;
    const size_t total = wpr * (size_t)height;
    for (size_t i = bk.idx.x * (size_t)bk.nt + bk.t; i < total; i += (size_t)bk.dim.x * bk.nt) {
        const size_t r = i / wpr, w = i - r * wpr;
        reinterpret_cast<uint4*>(dst + r * dpitch)[w] = reinterpret_cast<const uint4*>(src + r * spitch)[w];
    }
}

}  // namespace mlsdc
