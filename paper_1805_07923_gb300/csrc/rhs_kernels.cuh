// The three stage kernels of one explicit right-hand-side evaluation F_E
// (Sec. 2, Sec. 3, Sec. 4.1), templated on the arithmetic type T of the
// Legendre sums and FFTs: T = double (float64 path) or float (mixed
// precision).  The state is always float64 on input and F_E float64 on
// output.
//
//   k_synth_rhs<T>  per (m, 32 northern latitudes), 4 warps splitting the
//                   degrees n: Legendre sums split in even/odd n - m so one
//                   pass serves a latitude and its southern mirror
//                   (P^m_n(-mu) = (-1)^(n-m) P^m_n(mu), H^m_n(-mu) =
//                   -(-1)^(n-m) H^m_n(mu)); writes the Fourier coefficients
//                   of zeta, Phi', U, V                  -> four_in[4][J][R+1]
//   k_grid_rhs<T>   per latitude: real inverse FFTs, the grid products
//                   A = (zeta+f)U, B = (zeta+f)V, C = Phi'U, D = Phi'V,
//                   E = (U^2+V^2)/(2(1-mu^2)), real forward FFTs, weights
//                   w/(1-mu^2)/I (A..D) or w/I (E)        -> four_out[5][..]
//   k_anal_rhs<T>   per (m, 32 degrees), latitude tiles split over warps:
//                   Gaussian sums with even/odd combinations, then in float64
//                   F_E = [-div(C,D), -div(A,B), curl(A,B) + n(n+1)/a^2 E].
// four_in is [field][J][R+1] (m contiguous).  four_out is [field][J][R+1]
// or, chosen per launch (FourStride), [field][R+1][J] (latitudes
// contiguous): the analysis kernels work per m over latitudes and then read
// whole cache lines, while the FFT kernel, one latitude per CTA, writes its
// row with stride J.  That costs the FFT kernel about 1 us at T170 and pays
// only when a launch carries several members (measured on GB300: from three).
#pragma once

#include <type_traits>

#include "async_copy.cuh"
#include "complex.cuh"
#include "convert.cuh"
#include "internal.h"

namespace mlsdc {

constexpr int kSynthWarps = 4;

// Element strides of latitude j and wavenumber m in one field of four_out:
// (R + 1, 1) m-contiguous or (1, J) latitude-contiguous.
struct FourStride {
    int sj, sm;
    __host__ __device__ size_t at(int j, int m) const { return (size_t)j * sj + (size_t)m * sm; }
};
inline FourStride four_out_layout(int J, int R, bool lat_contig) {
    return lat_contig ? FourStride{1, J} : FourStride{R + 1, 1};
}
// float32 path: latitude-contiguous four_out from this many members per launch
constexpr int kLatContigMembers = 3;
constexpr int kAnalWarpsMax = 4;

// Ensemble batching: blockIdx.y selects the member, and each array advances
// by its member stride (in complex elements).  One member: all strides unused.
struct MemberStrides {
    size_t state, four_in, four_out, fe;
};

template <class T>
inline size_t synth_smem(int R) {
    const size_t coef = sizeof(C_t<T>) * 4 * (R + 1);
    const size_t red = sizeof(C_t<T>) * kSynthWarps * 6 * 32;
    return coef > red ? coef : red;
}
// The float32 synthesis with its tables streamed by TMA: the coefficient /
// reduction area, 128 bytes of alignment slack, the P and H rows of one work
// item (up to R + 1 rows of 32 latitudes each, in boxes of kSynBoxRows rows),
// and one mbarrier per box.
__host__ __device__ inline int synth_boxes(int R) { return (R + 1 + kSynBoxRows - 1) / kSynBoxRows; }
__host__ __device__ inline size_t synth_coef_bytes(int R) {
    const size_t coef = sizeof(float2) * 4 * (size_t)(R + 1), red = sizeof(float2) * kSynthWarps * 6 * 32;
    return ((coef > red ? coef : red) + 127) / 128 * 128;
}
inline size_t synth_tma_smem(int R) {
    return synth_coef_bytes(R) + 128 + (size_t)2 * synth_boxes(R) * kSynBoxRows * 32 * sizeof(float) +
           8 * (size_t)synth_boxes(R);
}

// U^m = (1/a) sum_n [ i m chi P - psi H ],  V^m = (1/a) sum_n [ i m psi P + chi H ]
// with psi, chi = -a^2/(n(n+1)) (zeta, delta) (Helmholtz, Sec. 2).
// With TMA (float32 only) the work item's table rows come into
// shared memory by TMA (maps: boxes of min(32, J2) latitudes x kSynBoxRows
// rows, one mbarrier per box of P and H rows), all issued before the
// coefficients are read; the warps wait for each box as their degrees reach
// it (bounded; a wait that gives up records kErrTmaTimeout in *err).
// Otherwise every thread reads its latitude's table entries from global
// memory.  Both forms form the same sums in the same order.
template <class T, bool TMA>
__device__ __forceinline__ void b_synth_rhs(const Blk& bk, const SynMaps& maps, int* err, const double2* state,
                                            const T* P, const T* H, const T* invnn, const Chunk* chunks, int R,
                                            int J2, int nc, double na2, double ia, C_t<T>* four, MemberStrides ms) {
    using C = C_t<T>;
    C* sc = reinterpret_cast<C*>(bk.smem);  // [nm][4]: zeta, Phi', chi, psi; reused for the reduction
    const Chunk ch = chunks[bk.idx.x];
    const int m = ch.m;
    const int nm = R + 1 - m;
    const int off = m * (R + 1) - m * (m - 1) / 2;
    constexpr bool tma = TMA && std::is_same<T, float>::value;
    const int bw = J2 < 32 ? J2 : 32;  // latitudes per table row in shared memory
    const int nbox = (nm + kSynBoxRows - 1) / kSynBoxRows;
    float* tP = reinterpret_cast<float*>(((uintptr_t)(bk.smem + synth_coef_bytes(R)) + 127) & ~(uintptr_t)127);
    float* tH = tP + (size_t)synth_boxes(R) * kSynBoxRows * 32;
    uint64_t* bars = reinterpret_cast<uint64_t*>(tH + (size_t)synth_boxes(R) * kSynBoxRows * 32);
    if (tma && bk.t == 0) {  // the tables are constant: their loads may start before the previous kernel ends
        for (int i = 0; i < nbox; ++i) mbar_init(sa(&bars[i]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int i = 0; i < nbox; ++i) {
            mbar_expect_tx(sa(&bars[i]), (uint32_t)(2 * kSynBoxRows * bw * sizeof(float)));
            tma_load_2d(sa(tP + (size_t)i * kSynBoxRows * bw), &maps.P, ch.start, off + i * kSynBoxRows,
                        sa(&bars[i]));
            tma_load_2d(sa(tH + (size_t)i * kSynBoxRows * bw), &maps.H, ch.start, off + i * kSynBoxRows,
                        sa(&bars[i]));
        }
    }
    pdl_wait();
    pdl_launch();
    state += bk.idx.y * ms.state;
    four += bk.idx.y * ms.four_in;
    for (int k = bk.t; k < nm; k += bk.nt) {
        // psi, chi = -a^2/(n(n+1)) (zeta, delta), the factor from the plan's table
        const T s = T(na2) * invnn[m + k];
        const double2 ph = state[off + k];
        const double2 ze = state[nc + off + k];
        const double2 de = state[2 * nc + off + k];
        sc[4 * k + 0] = mkc(T(ze.x), T(ze.y));
        sc[4 * k + 1] = mkc(T(ph.x), T(ph.y));
        sc[4 * k + 2] = mkc(T(de.x) * s, T(de.y) * s);
        sc[4 * k + 3] = mkc(T(ze.x) * s, T(ze.y) * s);
    }
    bk.sync();
    const int lane = bk.t & 31;
    const int wid = bk.t >> 5;
    const int j = ch.start + lane;
    const bool live = j < J2;
    const C zero = mkc(T(0), T(0));
    // this warp sums k = wid, wid + 4, ...: one parity (wid & 1) only
    C az = zero, ap = zero, axP = zero, asP = zero, asH = zero, axH = zero;
    if (tma) {
        const float* Pm = tP + lane;
        const float* Hm = tH + lane;
        for (int i = 0; i < nbox; ++i) {
            if (!mbar_wait(sa(&bars[i]), 0)) {
                atomicExch(err, kErrTmaTimeout);
                break;
            }
            if (!live) continue;
            const int k1 = min(nm, (i + 1) * kSynBoxRows);
            // this warp's degrees in the box: k = wid mod kSynthWarps
#pragma unroll 8
            for (int k = i * kSynBoxRows + wid; k < k1; k += kSynthWarps) {
                const T p = Pm[k * bw], h = Hm[k * bw];
                const C z = sc[4 * k], f = sc[4 * k + 1], x = sc[4 * k + 2], s = sc[4 * k + 3];
                cfma(az, p, z);
                cfma(ap, p, f);
                cfma(axP, p, x);
                cfma(asP, p, s);
                cfma(asH, h, s);
                cfma(axH, h, x);
            }
        }
    } else if (live) {
        const T* Pm = P + (size_t)off * J2 + j;
        const T* Hm = H + (size_t)off * J2 + j;
#pragma unroll 8
        for (int k = wid; k < nm; k += kSynthWarps) {
            const T p = Pm[(size_t)k * J2], h = Hm[(size_t)k * J2];
            const C z = sc[4 * k], f = sc[4 * k + 1], x = sc[4 * k + 2], s = sc[4 * k + 3];
            cfma(az, p, z);
            cfma(ap, p, f);
            cfma(axP, p, x);
            cfma(asP, p, s);
            cfma(asH, h, s);
            cfma(axH, h, x);
        }
    }
    bk.sync();  // coefficient table no longer needed: reuse it for the partial sums
    // (every thread's waits are over: a block of the persistent kernel retires the barriers)
    if (tma && bk.persist && bk.t == 0)
        for (int i = 0; i < nbox; ++i) mbar_inval(sa(&bars[i]));
    C* red = sc;      // [kSynthWarps][6][32]
    red[(wid * 6 + 0) * 32 + lane] = az;
    red[(wid * 6 + 1) * 32 + lane] = ap;
    red[(wid * 6 + 2) * 32 + lane] = axP;
    red[(wid * 6 + 3) * 32 + lane] = asP;
    red[(wid * 6 + 4) * 32 + lane] = asH;
    red[(wid * 6 + 5) * 32 + lane] = axH;
    bk.sync();
    if (wid != 0 || !live) return;
    C e[6], o[6];
    for (int q = 0; q < 6; ++q) {
        e[q] = cadd(red[(0 * 6 + q) * 32 + lane], red[(2 * 6 + q) * 32 + lane]);
        o[q] = cadd(red[(1 * 6 + q) * 32 + lane], red[(3 * 6 + q) * 32 + lane]);
    }
    const T iaT = T(ia);
    const T dm = T(m);
    const int J = 2 * J2;
    const int jS = J - 1 - j;
    const size_t fs = (size_t)J * (R + 1);
    const size_t iN = (size_t)j * (R + 1) + m, iS = (size_t)jS * (R + 1) + m;
    // north: P-sums e + o, H-sums e + o; south: P-sums e - o, H-sums o - e
    const C zN = cadd(e[0], o[0]), zS = csub(e[0], o[0]);
    const C pN = cadd(e[1], o[1]), pS = csub(e[1], o[1]);
    const C xPN = cadd(e[2], o[2]), xPS = csub(e[2], o[2]);
    const C sPN = cadd(e[3], o[3]), sPS = csub(e[3], o[3]);
    const C sHN = cadd(e[4], o[4]), sHS = csub(o[4], e[4]);
    const C xHN = cadd(e[5], o[5]), xHS = csub(o[5], e[5]);
    four[0 * fs + iN] = zN;
    four[0 * fs + iS] = zS;
    four[1 * fs + iN] = pN;
    four[1 * fs + iS] = pS;
    four[2 * fs + iN] = cscale(csub(cim(dm, xPN), sHN), iaT);
    four[2 * fs + iS] = cscale(csub(cim(dm, xPS), sHS), iaT);
    four[3 * fs + iN] = cscale(cadd(cim(dm, sPN), xHN), iaT);
    four[3 * fs + iS] = cscale(cadd(cim(dm, sPS), xHS), iaT);
}
template <class T, bool TMA>
__global__ void __launch_bounds__(32 * kSynthWarps) k_synth_rhs(const __grid_constant__ SynMaps maps,
                                                                int* __restrict__ err,
                                                                const double2* __restrict__ state,
                                                                const T* __restrict__ P, const T* __restrict__ H,
                                                                const T* __restrict__ invnn,
                                                                const Chunk* __restrict__ chunks, int R, int J2,
                                                                int nc, double na2, double ia, C_t<T>* __restrict__ four,
                                                                MemberStrides ms) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    b_synth_rhs<T, TMA>(hw_blk(smem_raw), maps, err, state, P, H, invnn, chunks, R, J2, nc, na2, ia, four, ms);
}

// LPB latitudes per CTA (1, or 2 adjacent ones for latitude-contiguous
// output: the two values of a (field, m) pair then leave in one store).
// stabg: the plan's stage-twiddle table (fft4_stage_twiddles of tw, I/2 - 1
// entries, formed once per plan by k_stage_twiddles), copied into shared
// memory with its load issued before the packing loads so that the two
// latencies overlap.
template <class T, int LPB>
__device__ __forceinline__ void b_grid_rhs(const Blk& bk, const C_t<T>* four_in, C_t<T>* four_out, const T* lat,
                                           const C_t<T>* __restrict__ tw, const C_t<T>* __restrict__ stabg, int R,
                                           int I, int logI, int J, double two_omega, MemberStrides ms,
                                           FourStride fx) {
    using C = C_t<T>;
    // [LPB][4][I/2]: zeta, Phi', U, V packed rows; then [LPB][5][I/2]: A..E; then the twiddles
    C* sx = reinterpret_cast<C*>(bk.smem);
    const int Hn = I >> 1, logH = logI - 1;
    C* stab = sx + 9 * LPB * Hn;  // stage twiddles (I/2 - 1 entries)
    const int nst = Hn - 1;
    const bool one_each = nst <= (int)bk.nt;  // one entry per thread: held in a register over the packing loop
    C twr = mkc(T(0), T(0));
    if (one_each) {
        if ((int)bk.t < nst) twr = stabg[bk.t];
    } else {
        for (int e = bk.t; e < nst; e += bk.nt) stab[e] = stabg[e];
    }
    const int j0 = bk.idx.x * LPB;
    // lat[j] = (mu, 1/(1-mu^2), w/((1-mu^2) I), w/I): no float64 division
    // here.  A constant table: with one latitude per CTA (launches of one or
    // two members, few CTAs) it is loaded ahead of its uses between the FFT
    // passes, taking its latency off the chain of barriers; with two (batched
    // launches, many CTAs per SM) the extra registers measured slower, and it
    // is read where it is used.
    T latv[LPB][4];
    if (LPB == 1) {
#pragma unroll
        for (int q = 0; q < 4; ++q) latv[0][q] = lat[4 * j0 + q];
    }
    pdl_wait();
    pdl_launch();
    four_in += bk.idx.y * ms.four_in;
    four_out += bk.idx.y * ms.four_out;
    const size_t fs = (size_t)J * (R + 1);
    for (int t = bk.t; t < 4 * LPB * Hn; t += bk.nt) {
        const int r = t >> logH, k = t & (Hn - 1);  // row r = 4 l + f
        const int l = r >> 2, f = r & 3;
        sx[r * Hn + swz(k)] = irfft_pack(four_in + f * fs + (size_t)(j0 + l) * (R + 1), k, R, Hn, tw);
    }
    if (one_each && (int)bk.t < nst) stab[bk.t] = twr;
    bk.sync();
    // inverse by decimation in frequency: slot q now holds the longitude pair
    // at the digit-reversed position of q
    fft4_dif(bk, sx, 4 * LPB, Hn, logH, stab, true);
    C* y = sx + 4 * LPB * Hn;
    T fl[LPB], rcl[LPB];
#pragma unroll
    for (int l = 0; l < LPB; ++l) {
        if (LPB > 1) {
            latv[l][0] = lat[4 * (j0 + l)];
            latv[l][1] = lat[4 * (j0 + l) + 1];
        }
        fl[l] = T(two_omega) * latv[l][0];
        rcl[l] = latv[l][1];
    }
    for (int t = bk.t; t < LPB * Hn; t += bk.nt) {
        const int l = LPB == 1 ? 0 : t >> logH;
        const C* xl = sx + 4 * l * Hn;
        C* yl = y + 5 * l * Hn;
        const T f = LPB == 1 ? fl[0] : (l ? fl[LPB - 1] : fl[0]);
        const T rc = LPB == 1 ? rcl[0] : (l ? rcl[LPB - 1] : rcl[0]);
        // .x and .y hold the two longitudes of one packed pair; products are
        // pointwise, so they stay in the same (permuted, swizzled) slot
        const int q = swz(t & (Hn - 1));
        const C z = xl[q], p = xl[Hn + q], u = xl[2 * Hn + q], v = xl[3 * Hn + q];
        const T zf0 = z.x + f, zf1 = z.y + f;
        yl[q] = mkc(zf0 * u.x, zf1 * u.y);                                        // A
        yl[Hn + q] = mkc(zf0 * v.x, zf1 * v.y);                                   // B
        yl[2 * Hn + q] = mkc(p.x * u.x, p.y * u.y);                               // C
        yl[3 * Hn + q] = mkc(p.x * v.x, p.y * v.y);                               // D
        yl[4 * Hn + q] = mkc(T(0.5) * (u.x * u.x + v.x * v.x) * rc,               // E
                             T(0.5) * (u.y * u.y + v.y * v.y) * rc);
    }
    bk.sync();
    // forward by decimation in time from the digit-reversed slots: natural order out
    fft4_dit(bk, y, 5 * LPB, Hn, logH, stab, false);
    T sAD[LPB], sE[LPB];  // w/((1-mu^2) I) for A..D, w/I for E
#pragma unroll
    for (int l = 0; l < LPB; ++l) {
        if (LPB > 1) {
            latv[l][2] = lat[4 * (j0 + l) + 2];
            latv[l][3] = lat[4 * (j0 + l) + 3];
        }
        sAD[l] = latv[l][2];
        sE[l] = latv[l][3];
    }
    for (int t = bk.t; t < 5 * (R + 1); t += bk.nt) {
        const int fld = t / (R + 1);
        const int m = t - fld * (R + 1);
        if (LPB == 1) {
            const C X = rfft_unpack_sw(y + fld * Hn, m, Hn, tw);
            four_out[(size_t)fld * fs + fx.at(j0, m)] = cscale(X, fld < 4 ? sAD[0] : sE[0]);
        } else {
            C X[LPB];
#pragma unroll
            for (int l = 0; l < LPB; ++l)
                X[l] = cscale(rfft_unpack_sw(y + (5 * l + fld) * Hn, m, Hn, tw), fld < 4 ? sAD[l] : sE[l]);
            C* dst = four_out + (size_t)fld * fs + fx.at(j0, m);
            if (sizeof(C) == 8 && fx.sj == 1) {
                // two adjacent latitudes: one 16-byte store (j0, J even: aligned)
                *reinterpret_cast<float4*>(dst) = make_float4(X[0].x, X[0].y, X[1].x, X[1].y);
            } else {
#pragma unroll
                for (int l = 0; l < LPB; ++l) dst[(size_t)l * fx.sj] = X[l];
            }
        }
    }
}
template <class T, int LPB>
__global__ void __launch_bounds__(256) k_grid_rhs(const C_t<T>* __restrict__ four_in, C_t<T>* __restrict__ four_out,
                                                  const T* __restrict__ lat, const C_t<T>* __restrict__ tw,
                                                  const C_t<T>* __restrict__ stabg, int R, int I, int logI, int J,
                                                  double two_omega, MemberStrides ms, FourStride fx) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    b_grid_rhs<T, LPB>(hw_blk(smem_raw), four_in, four_out, lat, tw, stabg, R, I, logI, J, two_omega, ms, fx);
}

// The stage-twiddle table of a plan (fft4_stage_twiddles into global memory),
// formed once by one CTA.
template <class C>
__global__ void k_stage_twiddles(C* __restrict__ tab, const C* __restrict__ tw, int N, int logN, int I) {
    fft4_stage_twiddles(hw_blk(nullptr), tab, tw, N, logN, I);
}

// div(X,Y)^m_n = (1/a) sum_j [ i m X' P - Y' H ], curl(X,Y)^m_n = (1/a) sum_j [ i m Y' P + X' H ]
// with X', Y' the weighted Fourier coefficients (integration by parts of the
// mu-derivatives); E^m_n = sum_j E' P.  With two_omega_lin != 0 the grid
// products were formed without f and the Coriolis part is added here exactly.
// Products and sums rounded as written (never contracted by the compiler),
// in float32 or float64.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// F_E's rows from the analysis sums of one coefficient (m, n) (Sec. 2):
// f0 = -div(C, D), f1 = -div(A, B), f2 = curl(A, B) + n(n+1)/a^2 E, with
// div(X, Y) = (1/a)(i m X_P - Y_H) and curl(X, Y) = (1/a)(i m Y_P + X_H),
// in the sums' type T with every operation rounded explicitly, so that each
// kernel and the persistent kernel's copy of it round alike; then widened to
// float64 (exactly).  s*: the P-table sums, h*: the H-table sums.
template <class C, class T>
__device__ __forceinline__ void fe_rows(C sC, C sA, C sB, C sE, C hD, C hB, C hA, T dm, T ia, int n, double2& f0,
                                        double2& f1, double2& f2) {
    const T dCDx = mul_rn(fma_rn(-dm, sC.y, -hD.x), ia), dCDy = mul_rn(fma_rn(dm, sC.x, -hD.y), ia);
    const T dABx = mul_rn(fma_rn(-dm, sA.y, -hB.x), ia), dABy = mul_rn(fma_rn(dm, sA.x, -hB.y), ia);
    const T cABx = mul_rn(fma_rn(-dm, sB.y, hA.x), ia), cABy = mul_rn(fma_rn(dm, sB.x, hA.y), ia);
    const T lap = mul_rn(mul_rn(mul_rn(T(n), T(n + 1)), ia), ia);
    f0 = make_double2(f64_of(-dCDx), f64_of(-dCDy));
    f1 = make_double2(f64_of(-dABx), f64_of(-dABy));
    f2 = make_double2(f64_of(fma_rn(lap, sE.x, cABx)), f64_of(fma_rn(lap, sE.y, cABy)));
}

constexpr int kAnalTW = 32;  // latitudes per tile of the CUDA-core analysis
// shared memory of the CUDA-core analysis: per warp [lat][field A..E][even,
// odd] sums, then the partial sums of warps 1.. for the reduction
template <class T>
constexpr size_t anal_smem_bytes() {
    return sizeof(C_t<T>) * ((size_t)kAnalWarpsMax * kAnalTW * 5 * 2 + (size_t)(kAnalWarpsMax - 1) * 7 * 32);
}

template <class T>
__device__ __forceinline__ void b_anal_rhs(const Blk& bk, const C_t<T>* four_out, const T* P, const T* H,
                                           const Chunk* chunks, int R, int J2, int nc, double ia, double2* FE,
                                           const double2* state, double two_omega_lin, const double* cor,
                                           MemberStrides ms, FourStride fx) {
    using C = C_t<T>;
    constexpr int TW = kAnalTW;
    pdl_wait();
    pdl_launch();
    four_out += bk.idx.y * ms.four_out;
    FE += bk.idx.y * ms.fe;
    state += bk.idx.y * ms.state;
    C(*sG)[TW][5][2] = reinterpret_cast<C(*)[TW][5][2]>(bk.smem);  // [warp][lat][field][even, odd]
    C(*red)[7][32] = reinterpret_cast<C(*)[7][32]>(bk.smem + sizeof(C) * kAnalWarpsMax * TW * 5 * 2);
    const Chunk ch = chunks[bk.idx.x];
    const int m = ch.m;
    const int nm = R + 1 - m;
    const int off = m * (R + 1) - m * (m - 1) / 2;
    const int k0 = ch.start;
    const int lane = bk.t & 31;
    const int wid = bk.t >> 5;
    const int nw = bk.nt >> 5;
    const int k = k0 + lane;
    const int par = k & 1;
    const int J = 2 * J2;
    const size_t fs = (size_t)J * (R + 1);
    const bool live = lane < nm - k0;
    const C zero = mkc(T(0), T(0));
    C aC = zero, aA = zero, aB = zero, aE = zero, hD = zero, hB = zero, hA = zero;
    const T* Prow = P + (size_t)(off + (live ? k : k0)) * J2;
    const T* Hrow = H + (size_t)(off + (live ? k : k0)) * J2;
    for (int jt = wid * TW; jt < J2; jt += nw * TW) {
        const int nl = min(TW, J2 - jt);
        if (lane < nl) {
            const int jn = jt + lane, js = J - 1 - jn;  // consecutive lanes: consecutive latitudes
            for (int f = 0; f < 5; ++f) {
                const C gN = four_out[(size_t)f * fs + fx.at(jn, m)];
                const C gS = four_out[(size_t)f * fs + fx.at(js, m)];
                sG[wid][lane][f][0] = cadd(gN, gS);
                sG[wid][lane][f][1] = csub(gN, gS);
            }
        }
        __syncwarp();
        if (live) {
#pragma unroll 8
            for (int jj = 0; jj < nl; ++jj) {
                const T p = Prow[jt + jj], h = Hrow[jt + jj];
                cfma(aC, p, sG[wid][jj][2][par]);
                cfma(aA, p, sG[wid][jj][0][par]);
                cfma(aB, p, sG[wid][jj][1][par]);
                cfma(aE, p, sG[wid][jj][4][par]);
                cfma(hD, h, sG[wid][jj][3][par ^ 1]);
                cfma(hB, h, sG[wid][jj][1][par ^ 1]);
                cfma(hA, h, sG[wid][jj][0][par ^ 1]);
            }
        }
        __syncwarp();
    }
    if (wid > 0) {
        red[wid - 1][0][lane] = aC;
        red[wid - 1][1][lane] = aA;
        red[wid - 1][2][lane] = aB;
        red[wid - 1][3][lane] = aE;
        red[wid - 1][4][lane] = hD;
        red[wid - 1][5][lane] = hB;
        red[wid - 1][6][lane] = hA;
    }
    bk.sync();
    if (wid != 0 || !live) return;
    // The sums of the other warps, then div, curl and the kinetic-energy
    // term in the working precision T: float64 on the float64 path; float32
    // on the mixed path, whose sums are float32 already (and float64 runs at
    // a small fraction of the float32 rate on this GPU).
    C s[7] = {aC, aA, aB, aE, hD, hB, hA};
    for (int w2 = 1; w2 < nw; ++w2)
        for (int q = 0; q < 7; ++q) s[q] = cadd(s[q], red[w2 - 1][q][lane]);
    const int n = m + k;
    double2 f0, f1, f2;
    fe_rows(s[0], s[1], s[2], s[3], s[4], s[5], s[6], T(m), T(ia), n, f0, f1, f2);
    if (two_omega_lin != 0.0) coriolis_add(state, cor, nc, R, m, n, off, two_omega_lin, f1, f2);
    if (m == 0) f0.y = f1.y = f2.y = 0.0;
    FE[off + k] = f0;
    FE[nc + off + k] = f1;
    FE[2 * nc + off + k] = f2;
}
template <class T>
__global__ void __launch_bounds__(32 * kAnalWarpsMax) k_anal_rhs(const C_t<T>* __restrict__ four_out,
                                                                 const T* __restrict__ P, const T* __restrict__ H,
                                                                 const Chunk* __restrict__ chunks, int R, int J2,
                                                                 int nc, double ia, double2* __restrict__ FE,
                                                                 const double2* __restrict__ state,
                                                                 double two_omega_lin, const double* __restrict__ cor,
                                                                 MemberStrides ms, FourStride fx) {
    __shared__ __align__(16) unsigned char sm[anal_smem_bytes<T>()];
    b_anal_rhs<T>(hw_blk(sm), four_out, P, H, chunks, R, J2, nc, ia, FE, state, two_omega_lin, cor, ms, fx);
}

// Launch helpers shared by both precisions.
template <class T>
inline size_t grid_smem(int I, int lpb = 1) {
    return sizeof(C_t<T>) * (9 * lpb + 1) * (size_t)(I / 2);  // nine rows per latitude and the twiddles
}
inline int anal_warps(int J2) {
    const int tiles = (J2 + 31) / 32;
    return tiles < kAnalWarpsMax ? tiles : kAnalWarpsMax;
}

}  // namespace mlsdc
