// Reverse mode of the MLSDC time step with respect to its initial state, for
// the geopotential misfit J = 1/2 ||Phi'(T) - Phi_t||^2 (Parseval norm,
// Sec. 3), with checkpointing.  All arithmetic is float64.
//
// Inner product: a state is the real vector of the (Re, Im) parts of its
// stored coefficients, <x, y> = sum Re(conj(x) y); Im of m = 0 is not a
// degree of freedom (the fields are real).  The transpose T^t of a real-linear
// map satisfies <y, T x> = <T^t y, x>.
//
// Only F_E is nonlinear.  A step is the fixed list of operations that
// build_mlsdc_ops produces (Algorithm 1); the adjoint walks that list
// backwards and applies each operation's transpose to adjoint buffers that
// mirror the forward ones, with F_E replaced by the transpose of its
// Jacobian at the recorded input ("tape").  Adjoint semantics of an
// operation y = op(x): x_bar += (d op / d x)^t y_bar, then y_bar = 0, since
// y was written (not accumulated) by the operation.
//
// The transpose of F_E'(x) (Sec. 2, Sec. 4.1; derivation of each line in the
// kernel comments):
//   k_synth_ad  per (m, 32 northern latitudes): Legendre sums of the state x
//               (zeta, Phi', U, V, as the forward) and of lambda:
//                 H_A = (1/a) sum [ i m P l_zeta + H l_delta ]
//                 H_B = (1/a) sum [ H l_zeta - i m P l_delta ]
//                 H_C = (1/a) sum i m P l_Phi,  H_D = (1/a) sum H l_Phi
//                 H_E = sum n(n+1)/a^2 P l_delta
//               times 1 (m = 0) or 1/2 (m >= 1)             -> four_in[9][J][R+1]
//   k_grid_ad   per latitude: inverse real FFTs of all nine; with
//               s = w_j / ((1 - mu^2) I), s_E = w_j / I the grid adjoints
//               A_b = s H_A, .., E_b = s_E H_E of the products
//               A = (zeta+f)U, B = (zeta+f)V, C = Phi'U, D = Phi'V,
//               E = (U^2+V^2)/(2(1-mu^2)) give
//                 zeta_b = A_b U + B_b V,  Phi_b = C_b U + D_b V,
//                 U_b = A_b (zeta+f) + C_b Phi' + E_b U/(1-mu^2),
//                 V_b = B_b (zeta+f) + D_b Phi' + E_b V/(1-mu^2);
//               forward real FFTs (unnormalised) times 1 (m = 0) or 2  -> four_out[4][J][R+1]
//   k_anal_ad   per (m, 32 degrees): Gaussian sums without weights,
//                 psi_b = (1/a) sum [ -H U_b - i m P V_b ],
//                 chi_b = (1/a) sum [ -i m P U_b + H V_b ],
//                 x_b += [ sum P Phi_b,  sum P zeta_b + s_n psi_b,  s_n chi_b ],
//               s_n = -a^2/(n(n+1)).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "complex.cuh"
#include "internal.h"
#include "rhs_kernels.cuh"
#include "sdc_internal.h"

namespace mlsdc {

constexpr int kAdSynthWarps = 4;
constexpr int kAdSums = 13;

// ---------------------------------------------------------------------------
// F_E'(x)^t

__global__ void __launch_bounds__(32 * kAdSynthWarps) k_synth_ad(const double2* __restrict__ x,
                                                                 const double2* __restrict__ lam,
                                                                 const double* __restrict__ P,
                                                                 const double* __restrict__ H,
                                                                 const double* __restrict__ invnn,
                                                                 const Chunk* __restrict__ chunks, int R, int J2,
                                                                 int nc, double a, double ia,
                                                                 double2* __restrict__ four) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2* sc = reinterpret_cast<double2*>(smem_raw);  // [nm][8], then the reduction
    const Chunk ch = chunks[blockIdx.x];
    const int m = ch.m;
    const int nm = R + 1 - m;
    const int off = m * (R + 1) - m * (m - 1) / 2;
    const double ia2 = ia * ia;
    for (int k = threadIdx.x; k < nm; k += blockDim.x) {
        const int n = m + k;
        const double s = -a * a * invnn[n];  // -a^2/(n(n+1)), 0 for n = 0
        const double2 ph = x[off + k], ze = x[nc + off + k], de = x[2 * nc + off + k];
        double2 lp = lam[off + k], lz = lam[nc + off + k], ld = lam[2 * nc + off + k];
        if (m == 0) lp.y = lz.y = ld.y = 0.0;  // Im of m = 0 is not a degree of freedom
        const double lap = n * (n + 1.0) * ia2;
        double2* c = sc + 8 * k;
        c[0] = ze;
        c[1] = ph;
        c[2] = make_double2(de.x * s, de.y * s);  // chi
        c[3] = make_double2(ze.x * s, ze.y * s);  // psi
        c[4] = lp;
        c[5] = lz;
        c[6] = ld;
        c[7] = make_double2(ld.x * lap, ld.y * lap);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int j = ch.start + lane;
    const bool live = j < J2;
    double2 acc[kAdSums];
#pragma unroll
    for (int q = 0; q < kAdSums; ++q) acc[q] = make_double2(0.0, 0.0);
    if (live) {
        const double* Pm = P + (size_t)off * J2 + j;
        const double* Hm = H + (size_t)off * J2 + j;
#pragma unroll 4
        for (int k = wid; k < nm; k += kAdSynthWarps) {  // one parity of n - m per warp
            const double p = Pm[(size_t)k * J2], h = Hm[(size_t)k * J2];
            const double2* c = sc + 8 * k;
            cfma(acc[0], p, c[0]);   // P zeta
            cfma(acc[1], p, c[1]);   // P Phi'
            cfma(acc[2], p, c[2]);   // P chi
            cfma(acc[3], p, c[3]);   // P psi
            cfma(acc[4], h, c[3]);   // H psi
            cfma(acc[5], h, c[2]);   // H chi
            cfma(acc[6], p, c[4]);   // P l_Phi
            cfma(acc[7], h, c[4]);   // H l_Phi
            cfma(acc[8], p, c[5]);   // P l_zeta
            cfma(acc[9], h, c[5]);   // H l_zeta
            cfma(acc[10], p, c[6]);  // P l_delta
            cfma(acc[11], h, c[6]);  // H l_delta
            cfma(acc[12], p, c[7]);  // P n(n+1)/a^2 l_delta
        }
    }
    __syncthreads();
    double2* red = sc;  // [warps][sums][32]
    for (int q = 0; q < kAdSums; ++q) red[(wid * kAdSums + q) * 32 + lane] = acc[q];
    __syncthreads();
    if (wid != 0 || !live) return;
    // even n - m: warps 0, 2; odd: warps 1, 3.  North = e + o for P and H;
    // south = e - o for P, o - e for H (parity of P and H in mu).
    const bool isH[kAdSums] = {false, false, false, false, true, true, false, true, false, true, false, true, false};
    double2 N[kAdSums], S[kAdSums];
    for (int q = 0; q < kAdSums; ++q) {
        const double2 e = cadd(red[(0 * kAdSums + q) * 32 + lane], red[(2 * kAdSums + q) * 32 + lane]);
        const double2 o = cadd(red[(1 * kAdSums + q) * 32 + lane], red[(3 * kAdSums + q) * 32 + lane]);
        N[q] = cadd(e, o);
        S[q] = isH[q] ? csub(o, e) : csub(e, o);
    }
    const double dm = (double)m;
    const double cm = m == 0 ? 1.0 : 0.5;  // transpose of the Hermitian inverse FFT
    const int J = 2 * J2;
    const size_t fs = (size_t)J * (R + 1);
    for (int hs = 0; hs < 2; ++hs) {
        const double2* s = hs == 0 ? N : S;
        const size_t row = (size_t)(hs == 0 ? j : J - 1 - j) * (R + 1) + m;
        four[0 * fs + row] = s[0];
        four[1 * fs + row] = s[1];
        four[2 * fs + row] = cscale(csub(cim(dm, s[2]), s[4]), ia);            // U
        four[3 * fs + row] = cscale(cadd(cim(dm, s[3]), s[5]), ia);            // V
        four[4 * fs + row] = cscale(cadd(cim(dm, s[8]), s[11]), ia * cm);      // H_A
        four[5 * fs + row] = cscale(csub(s[9], cim(dm, s[10])), ia * cm);      // H_B
        four[6 * fs + row] = cscale(cim(dm, s[6]), ia * cm);                   // H_C
        four[7 * fs + row] = cscale(s[7], ia * cm);                            // H_D
        four[8 * fs + row] = cscale(s[12], cm);                                // H_E
    }
}

__global__ void __launch_bounds__(256) k_grid_ad(const double2* __restrict__ four_in, double2* __restrict__ four_out,
                                                 const double* __restrict__ lat, const double2* __restrict__ tw,
                                                 int R, int I, int logI, int J, double two_omega) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2* sx = reinterpret_cast<double2*>(smem_raw);  // [9][I/2], then [I/2] twiddles
    const int j = blockIdx.x;
    const int Hn = I >> 1, logH = logI - 1;
    double2* stab = sx + 9 * Hn;
    const Blk bk = hw_blk(smem_raw);
    fft4_stage_twiddles(bk, stab, tw, Hn, logH, I);
    const size_t fs = (size_t)J * (R + 1);
    for (int t = threadIdx.x; t < 9 * Hn; t += blockDim.x) {
        const int f = t >> logH, k = t & (Hn - 1);
        sx[f * Hn + swz(k)] = irfft_pack(four_in + f * fs + (size_t)j * (R + 1), k, R, Hn, tw);
    }
    __syncthreads();
    fft4_dif(bk, sx, 9, Hn, logH, stab, true);
    // lat[j] = (mu, 1/(1-mu^2), w/((1-mu^2) I), w/I)
    const double f = two_omega * lat[4 * j];
    const double rc = lat[4 * j + 1];
    const double sAD = lat[4 * j + 2], sE = lat[4 * j + 3];
    for (int q0 = threadIdx.x; q0 < Hn; q0 += blockDim.x) {
        const int q = swz(q0);
        double2 v9[9];
        for (int k = 0; k < 9; ++k) v9[k] = sx[k * Hn + q];
        // .x and .y are two longitudes of one packed pair: pointwise in both
        double o[4][2];
        for (int h = 0; h < 2; ++h) {
            const double z = h ? v9[0].y : v9[0].x, p = h ? v9[1].y : v9[1].x;
            const double u = h ? v9[2].y : v9[2].x, v = h ? v9[3].y : v9[3].x;
            const double Ab = sAD * (h ? v9[4].y : v9[4].x), Bb = sAD * (h ? v9[5].y : v9[5].x);
            const double Cb = sAD * (h ? v9[6].y : v9[6].x), Db = sAD * (h ? v9[7].y : v9[7].x);
            const double Eb = sE * (h ? v9[8].y : v9[8].x);
            const double zf = z + f;
            o[0][h] = Ab * u + Bb * v;                         // zeta_b
            o[1][h] = Cb * u + Db * v;                         // Phi_b
            o[2][h] = Ab * zf + Cb * p + Eb * u * rc;          // U_b
            o[3][h] = Bb * zf + Db * p + Eb * v * rc;          // V_b
        }
        for (int k = 0; k < 4; ++k) sx[k * Hn + q] = make_double2(o[k][0], o[k][1]);
    }
    __syncthreads();
    fft4_dit(bk, sx, 4, Hn, logH, stab, false);
    for (int t = threadIdx.x; t < 4 * (R + 1); t += blockDim.x) {
        const int fld = t / (R + 1);
        const int m = t - fld * (R + 1);
        const double2 X = rfft_unpack_sw(sx + fld * Hn, m, Hn, tw);
        four_out[(size_t)fld * fs + (size_t)j * (R + 1) + m] = cscale(X, m == 0 ? 1.0 : 2.0);
    }
}

__global__ void __launch_bounds__(32 * kAnalWarpsMax) k_anal_ad(const double2* __restrict__ four,
                                                                const double* __restrict__ P,
                                                                const double* __restrict__ H,
                                                                const double* __restrict__ invnn,
                                                                const Chunk* __restrict__ chunks, int R, int J2,
                                                                int nc, double a, double ia,
                                                                double2* __restrict__ xb, double2* __restrict__ lam) {
    constexpr int TW = 32;
    __shared__ double2 sG[kAnalWarpsMax][TW][4][2];  // per warp: [lat][zeta_b, Phi_b, U_b, V_b][even, odd]
    __shared__ double2 red[kAnalWarpsMax - 1][6][32];
    const Chunk ch = chunks[blockIdx.x];
    const int m = ch.m;
    const int nm = R + 1 - m;
    const int off = m * (R + 1) - m * (m - 1) / 2;
    const int k0 = ch.start;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int k = k0 + lane;
    const int par = k & 1;
    const int J = 2 * J2;
    const size_t fs = (size_t)J * (R + 1);
    const bool live = lane < nm - k0;
    double2 aZ{0, 0}, aP{0, 0}, aU{0, 0}, aV{0, 0}, hU{0, 0}, hV{0, 0};
    const double* Prow = P + (size_t)(off + (live ? k : k0)) * J2;
    const double* Hrow = H + (size_t)(off + (live ? k : k0)) * J2;
    for (int jt = wid * TW; jt < J2; jt += nw * TW) {
        const int nl = min(TW, J2 - jt);
        for (int t = lane; t < nl * 4; t += 32) {
            const int jj = t >> 2, f = t & 3;
            const int jn = jt + jj, js = J - 1 - jn;
            const double2 gN = four[(size_t)f * fs + (size_t)jn * (R + 1) + m];
            const double2 gS = four[(size_t)f * fs + (size_t)js * (R + 1) + m];
            sG[wid][jj][f][0] = cadd(gN, gS);
            sG[wid][jj][f][1] = csub(gN, gS);
        }
        __syncwarp();
        if (live) {
#pragma unroll 8
            for (int jj = 0; jj < nl; ++jj) {
                const double p = Prow[jt + jj], h = Hrow[jt + jj];
                cfma(aZ, p, sG[wid][jj][0][par]);
                cfma(aP, p, sG[wid][jj][1][par]);
                cfma(aU, p, sG[wid][jj][2][par]);
                cfma(aV, p, sG[wid][jj][3][par]);
                cfma(hU, h, sG[wid][jj][2][par ^ 1]);
                cfma(hV, h, sG[wid][jj][3][par ^ 1]);
            }
        }
        __syncwarp();
    }
    if (wid > 0) {
        red[wid - 1][0][lane] = aZ;
        red[wid - 1][1][lane] = aP;
        red[wid - 1][2][lane] = aU;
        red[wid - 1][3][lane] = aV;
        red[wid - 1][4][lane] = hU;
        red[wid - 1][5][lane] = hV;
    }
    __syncthreads();
    if (wid != 0 || !live) return;
    for (int w2 = 1; w2 < nw; ++w2) {
        aZ = cadd(aZ, red[w2 - 1][0][lane]);
        aP = cadd(aP, red[w2 - 1][1][lane]);
        aU = cadd(aU, red[w2 - 1][2][lane]);
        aV = cadd(aV, red[w2 - 1][3][lane]);
        hU = cadd(hU, red[w2 - 1][4][lane]);
        hV = cadd(hV, red[w2 - 1][5][lane]);
    }
    const int n = m + k;
    const double dm = (double)m;
    const double sn = -a * a * invnn[n];  // -a^2/(n(n+1)), 0 for n = 0
    // psi_b = (1/a)(-H U_b - i m P V_b), chi_b = (1/a)(-i m P U_b + H V_b)
    const double2 psib = cscale(csub(make_double2(-hU.x, -hU.y), cim(dm, aV)), ia);
    const double2 chib = cscale(csub(hV, cim(dm, aU)), ia);
    double2 o0 = aP;
    double2 o1 = make_double2(aZ.x + sn * psib.x, aZ.y + sn * psib.y);
    double2 o2 = make_double2(sn * chib.x, sn * chib.y);
    if (m == 0) o0.y = o1.y = o2.y = 0.0;
    const size_t c = off + k;
    xb[c] = cadd(xb[c], o0);
    xb[nc + c] = cadd(xb[nc + c], o1);
    xb[2 * nc + c] = cadd(xb[2 * nc + c], o2);
    // the adjoint of F_E's output is consumed
    lam[c] = make_double2(0.0, 0.0);
    lam[nc + c] = make_double2(0.0, 0.0);
    lam[2 * nc + c] = make_double2(0.0, 0.0);
}

static size_t synth_ad_smem(int R) {
    return std::max(sizeof(double2) * kAdSynthWarps * kAdSums * 32, sizeof(double2) * 8 * (R + 1));
}
static size_t grid_ad_smem(int I) { return sizeof(double2) * 10 * (I / 2); }

// Shared-memory limits of the F_E adjoint kernels for a plan (outside any
// stream capture).
static mlsdc_status fe_adjoint_prepare(sh_plan_t p) {
    mlsdc_status s;
    if ((s = raise_smem_limit((const void*)k_synth_ad, synth_ad_smem(p->R))) != MLSDC_OK) return s;
    return raise_smem_limit((const void*)k_grid_ad, grid_ad_smem(p->I));
}

static mlsdc_status fe_adjoint(sh_plan_t p, const swe_params* prm, const double2* x, double2* lam, double2* xb,
                               cudaStream_t st, int64_t* launches) {
    const int R = p->R;
    const size_t ss = synth_ad_smem(R), gs = grid_ad_smem(p->I);
    k_synth_ad<<<p->n_synth, 32 * kAdSynthWarps, ss, st>>>(x, lam, p->d_P, p->d_H, p->d_invnn, p->d_synth, R, p->J2,
                                                          p->nc, prm->a, 1.0 / prm->a, p->d_four_in);
    MLSDC_LAUNCHED("k_synth_ad");
    k_grid_ad<<<p->J, 256, gs, st>>>(p->d_four_in, p->d_four_out, p->d_lat, p->d_tw, R, p->I, p->logI, p->J,
                                     2.0 * prm->omega);
    MLSDC_LAUNCHED("k_grid_ad");
    k_anal_ad<<<p->n_anal, 32 * anal_warps(p->J2), 0, st>>>(p->d_four_out, p->d_P, p->d_H, p->d_invnn, p->d_anal, R,
                                                           p->J2, p->nc, prm->a, 1.0 / prm->a, xb, lam);
    MLSDC_LAUNCHED("k_anal_ad");
    if (launches) *launches += 3;
    return MLSDC_OK;
}

// ---------------------------------------------------------------------------
// transposes of the linear operations of a step (single member)

__device__ __forceinline__ double2 axpy(double2 y, double s, double2 x) {
    return make_double2(fma(s, x.x, y.x), fma(s, x.y, y.y));
}

// dst += src; src = 0 (transpose of a copy src -> dst)
__global__ void k_acc_clear(double2* __restrict__ dst, double2* __restrict__ src, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        dst[i] = cadd(dst[i], src[i]);
        src[i] = make_double2(0.0, 0.0);
    }
}

// transpose of dst[k] = src, k < count
__global__ void k_bcast_ad(double2* __restrict__ srcb, double2* __restrict__ dstb, int n3, int count) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n3; c += gridDim.x * blockDim.x) {
        double2 s = srcb[c];
        for (int k = 0; k < count; ++k) {
            s = cadd(s, dstb[(size_t)k * n3 + c]);
            dstb[(size_t)k * n3 + c] = make_double2(0.0, 0.0);
        }
        srcb[c] = s;
    }
}

// transpose of F_I = [ -Phibar d + nu L p, nu L z, -L p + nu L d ]:
// [ nu L lp - L ld, nu L lz, -Phibar lp + nu L ld ]
__device__ __forceinline__ void implicit_rhs_t(double L, const Phys& ph, double2 lp, double2 lz, double2 ld,
                                               double2& p, double2& z, double2& d) {
    const double nl = ph.nu * L;
    p = make_double2(nl * lp.x - L * ld.x, nl * lp.y - L * ld.y);
    z = make_double2(nl * lz.x, nl * lz.y);
    d = make_double2(-ph.phibar * lp.x + nl * ld.x, -ph.phibar * lp.y + nl * ld.y);
}

// transpose of the implicit solve: (I - alpha F_I^t) y = g, with c = 1 - alpha nu L
// [[c, 0, alpha L], [0, c, 0], [alpha Phibar, 0, c]] y = g
// with the same two reciprocals r = solve_recips(L, alpha, ph) as the forward solve
__device__ __forceinline__ void implicit_solve_t(double L, double alpha, const Phys& ph, double2 r, double2 gp,
                                                 double2 gz, double2 gd, double2& p, double2& z, double2& d) {
    const double c = 1.0 - alpha * ph.nu * L;
    const double ic = r.x, den = r.y;
    z = make_double2(gz.x * ic, gz.y * ic);
    p = make_double2((c * gp.x - alpha * L * gd.x) * den, (c * gp.y - alpha * L * gd.y) * den);
    d = make_double2((gd.x - alpha * ph.phibar * p.x) * ic, (gd.y - alpha * ph.phibar * p.y) * ic);
}

__global__ void k_fi_ad(double2* __restrict__ xb, double2* __restrict__ Fb, const int* __restrict__ ndeg, int nc,
                        Phys ph) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
        const double n = ndeg[c];
        const double L = -n * (n + 1.0) * ph.inv_a2;
        double2 p, z, d;
        implicit_rhs_t(L, ph, Fb[c], Fb[nc + c], Fb[2 * nc + c], p, z, d);
        xb[c] = cadd(xb[c], p);
        xb[nc + c] = cadd(xb[nc + c], z);
        xb[2 * nc + c] = cadd(xb[2 * nc + c], d);
        Fb[c] = Fb[nc + c] = Fb[2 * nc + c] = make_double2(0.0, 0.0);
    }
}

// Transpose of k_sweep_node (node m+1 of one sweep):
//   b = Th[0] + sum_{j=1..m} dt (qE_j (FEn_j - FEo_j) + qI_j (FIn_j - FIo_j))
//       - dt qI_mm FIo_{m+1} + sum_{j=0..M} dt q_j (FIo_j + FEo_j) [+ tau_{m+1}]
//   Th[m+1] = solve(b);  FIn[m+1] = F_I(Th[m+1]);  (m = 0: FIn[0] = FIo[0], FEn[0] = FEo[0])
__global__ void k_node_ad(double2* Thb, double2* FIob, double2* FEob, double2* FInb, double2* FEnb, double2* taub,
                          const int* __restrict__ ndeg, const double2* __restrict__ recips, int nc, double dt,
                          NodeRow row, Phys ph) {
    const size_t node = (size_t)3 * nc;
    const int m = row.m;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
        if (m == 0)
            for (int f = 0; f < 3; ++f) {
                const size_t o = (size_t)f * nc + c;
                FIob[o] = cadd(FIob[o], FInb[o]);
                FEob[o] = cadd(FEob[o], FEnb[o]);
                FInb[o] = FEnb[o] = make_double2(0.0, 0.0);
            }
        const int nd = ndeg[c];
        const double n = nd;
        const double L = -n * (n + 1.0) * ph.inv_a2;
        const size_t om = (m + 1) * node + c;
        double2 gp, gz, gd;
        implicit_rhs_t(L, ph, FInb[om], FInb[om + nc], FInb[om + 2 * nc], gp, gz, gd);
        gp = cadd(gp, Thb[om]);
        gz = cadd(gz, Thb[om + nc]);
        gd = cadd(gd, Thb[om + 2 * nc]);
        for (int f = 0; f < 3; ++f) Thb[om + f * nc] = FInb[om + f * nc] = make_double2(0.0, 0.0);
        double2 b[3];
        implicit_solve_t(L, dt * row.qimm, ph, recips[nd], gp, gz, gd, b[0], b[1], b[2]);
        for (int f = 0; f < 3; ++f) {
            const size_t o = (size_t)f * nc + c;
            const double2 bb = b[f];
            Thb[o] = cadd(Thb[o], bb);
            for (int j = 1; j <= m; ++j) {
                const size_t oj = j * node + o;
                FEnb[oj] = axpy(FEnb[oj], dt * row.qe[j], bb);
                FEob[oj] = axpy(FEob[oj], -dt * row.qe[j], bb);
                FInb[oj] = axpy(FInb[oj], dt * row.qi[j], bb);
                FIob[oj] = axpy(FIob[oj], -dt * row.qi[j], bb);
            }
            const size_t o1 = (m + 1) * node + o;
            FIob[o1] = axpy(FIob[o1], -dt * row.qimm, bb);
            for (int j = 0; j <= row.M; ++j) {
                const size_t oj = j * node + o;
                FIob[oj] = axpy(FIob[oj], dt * row.q[j], bb);
                FEob[oj] = axpy(FEob[oj], dt * row.q[j], bb);
            }
            if (taub) taub[o1] = cadd(taub[o1], bb);
        }
    }
}

// transpose of Tc[i] = D(sum_j Pcf[i][j] Tf[j]), i in [i0, i1)
__global__ void k_restrict_ad(double2* __restrict__ Tfb, double2* __restrict__ Tcb, const int* __restrict__ c2f,
                              int ncf, int ncc, int nfn, int i0, int i1, TransferMat Pcf) {
    const int total = 3 * ncc;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int f = t / ncc, k = t - f * ncc;
        const size_t of = (size_t)f * ncf + c2f[k];
        double2 yb[kMaxNodes];
        for (int i = i0; i < i1; ++i) {
            yb[i] = Tcb[(size_t)i * 3 * ncc + t];
            Tcb[(size_t)i * 3 * ncc + t] = make_double2(0.0, 0.0);
        }
        for (int j = 0; j < nfn; ++j) {
            double2 acc = Tfb[(size_t)j * 3 * ncf + of];
            for (int i = i0; i < i1; ++i) acc = axpy(acc, Pcf.a[i * nfn + j], yb[i]);
            Tfb[(size_t)j * 3 * ncf + of] = acc;
        }
    }
}

// transpose of tau[i] = Tc[i] - dt sum_l Qc[i][l] (FIc+FEc)[l] - sum_j Pcf[i][j] Af[j],
// Af[j] = Tf[j] - dt sum_l Qf[j][l] (FIf+FEf)[l]  (fine values at the coarse modes)
// and of the saved copies Ts, FIs, FEs = Tc, FIc, FEc made in the same pass
__global__ void k_fas_ad(double2* __restrict__ Tfb, double2* __restrict__ FIfb, double2* __restrict__ FEfb,
                         double2* __restrict__ Tcb, double2* __restrict__ FIcb, double2* __restrict__ FEcb,
                         double2* __restrict__ taub, double2* __restrict__ Tsb, double2* __restrict__ FIsb,
                         double2* __restrict__ FEsb, const int* __restrict__ c2f, int ncf, int ncc, double dt,
                         FasArgs A) {
    const int total = 3 * ncc;
    const size_t nf3 = (size_t)3 * ncf, nc3 = (size_t)3 * ncc;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int f = t / ncc, k = t - f * ncc;
        const size_t of = (size_t)f * ncf + c2f[k];
        for (int i = 0; i < A.ncn; ++i) {
            const size_t oc = i * nc3 + t;
            Tcb[oc] = cadd(Tcb[oc], Tsb[oc]);
            FIcb[oc] = cadd(FIcb[oc], FIsb[oc]);
            FEcb[oc] = cadd(FEcb[oc], FEsb[oc]);
            Tsb[oc] = FIsb[oc] = FEsb[oc] = make_double2(0.0, 0.0);
        }
        double2 tb[kMaxNodes], Afb[kMaxNodes];
        for (int i = 0; i < A.ncn; ++i) {
            tb[i] = taub[i * nc3 + t];
            taub[i * nc3 + t] = make_double2(0.0, 0.0);
        }
        for (int i = 0; i < A.ncn; ++i) Tcb[i * nc3 + t] = cadd(Tcb[i * nc3 + t], tb[i]);
        for (int l = 0; l < A.ncn; ++l) {
            double2 s{0.0, 0.0};
            for (int i = 0; i < A.ncn; ++i) s = axpy(s, A.Qc[i * A.ncn + l], tb[i]);
            FIcb[l * nc3 + t] = axpy(FIcb[l * nc3 + t], -dt, s);
            FEcb[l * nc3 + t] = axpy(FEcb[l * nc3 + t], -dt, s);
        }
        for (int j = 0; j < A.nfn; ++j) {
            double2 s{0.0, 0.0};
            for (int i = 0; i < A.ncn; ++i) s = axpy(s, -A.Pcf[i * A.nfn + j], tb[i]);
            Afb[j] = s;
            Tfb[j * nf3 + of] = cadd(Tfb[j * nf3 + of], s);
        }
        for (int l = 0; l < A.nfn; ++l) {
            double2 s{0.0, 0.0};
            for (int j = 0; j < A.nfn; ++j) s = axpy(s, A.Qf[j * A.nfn + l], Afb[j]);
            FIfb[l * nf3 + of] = axpy(FIfb[l * nf3 + of], -dt, s);
            FEfb[l * nf3 + of] = axpy(FEfb[l * nf3 + of], -dt, s);
        }
    }
}

// transpose of X_f[m] += P(sum_i Pfc[m][i] (X_c[i] - X_s[i])), m = 1..Mf
__global__ void k_interp_ad(const double2* __restrict__ Tfb, const double2* __restrict__ FIfb,
                            const double2* __restrict__ FEfb, double2* __restrict__ Tcb, double2* __restrict__ FIcb,
                            double2* __restrict__ FEcb, double2* __restrict__ Tsb, double2* __restrict__ FIsb,
                            double2* __restrict__ FEsb, const int* __restrict__ c2f, int ncf, int ncc, int nfn,
                            int ncn, TransferMat Pfc) {
    const int total = 3 * ncc;
    const size_t nf3 = (size_t)3 * ncf, nc3 = (size_t)3 * ncc;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int f = t / ncc, k = t - f * ncc;
        const size_t of = (size_t)f * ncf + c2f[k];
        const double2* Xf[3] = {Tfb, FIfb, FEfb};
        double2* Xc[3] = {Tcb, FIcb, FEcb};
        double2* Xs[3] = {Tsb, FIsb, FEsb};
        for (int x = 0; x < 3; ++x)
            for (int i = 0; i < ncn; ++i) {
                double2 s{0.0, 0.0};
                for (int m = 1; m < nfn; ++m) s = axpy(s, Pfc.a[m * ncn + i], Xf[x][m * nf3 + of]);
                const size_t oc = i * nc3 + t;
                Xc[x][oc] = cadd(Xc[x][oc], s);
                Xs[x][oc] = make_double2(Xs[x][oc].x - s.x, Xs[x][oc].y - s.y);
            }
    }
}

__global__ void k_zero_m0_imag(double2* __restrict__ x, int R, int nc, int nf) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nf * (R + 1); t += gridDim.x * blockDim.x) {
        const int f = t / (R + 1), n = t - f * (R + 1);
        x[(size_t)f * nc + n].y = 0.0;  // m = 0 block: the first R + 1 coefficients
    }
}

// J = 1/2 sum w_m |Phi' - Phi_t|^2 (w_0 = 1, w_m = 2) and lambda = dJ/dx
// = [w_m (Phi' - Phi_t) (Im of m = 0 dropped), 0, 0]; one block, fixed order.
__global__ void __launch_bounds__(1024) k_misfit(const double2* __restrict__ x, const double2* __restrict__ target,
                                                 int R, int nc, double* __restrict__ J, double2* __restrict__ lam) {
    __shared__ double part[32];
    double acc = 0.0;
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
        const bool m0 = c <= R;
        const double wm = m0 ? 1.0 : 2.0;
        const double2 r = make_double2(x[c].x - target[c].x, m0 ? 0.0 : x[c].y - target[c].y);
        acc += wm * (r.x * r.x + r.y * r.y);
        lam[c] = make_double2(wm * r.x, wm * r.y);
        lam[nc + c] = make_double2(0.0, 0.0);
        lam[2 * nc + c] = make_double2(0.0, 0.0);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += part[w];
        *J = 0.5 * s;
    }
}

}  // namespace mlsdc

using namespace mlsdc;

// ---------------------------------------------------------------------------
// the adjoint driver

namespace {

struct Region {
    const double2* fwd;
    size_t n;  // complex values
    double2* adj;
};

}  // namespace

struct mlsdc_adjoint_s {
    mlsdc_t ml = nullptr;
    int n_steps = 0, every = 1, n_iter = 0, n_c = 0;
    double dt = 0.0;
    std::vector<Op> ops;
    size_t tape_step = 0;         // complex values of one step's tape
    double2* ck = nullptr;        // [n_ck][3][ncf] checkpoints (the state every `every` steps)
    double2* tape = nullptr;      // [every][tape_step]
    double2* work = nullptr;      // [3][ncf] the state the step operations run on
    double2* lam = nullptr;       // [3][ncf] adjoint of `work`
    double2* slab = nullptr;      // adjoint buffers of every level and transfer buffer
    size_t slab_n = 0;
    std::vector<Region> regions;
    bool have_forward = false;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t g_fwd = nullptr;
    std::vector<cudaGraphExec_t> g_tape, g_rev;
    int64_t launches_fwd = 0, launches_rev = 0;
};

namespace {

double2* adj_of(mlsdc_adjoint_t A, const double2* p) {
    if (!p) return nullptr;
    for (const Region& r : A->regions)
        if (p >= r.fwd && p < r.fwd + r.n) return r.adj + (p - r.fwd);
    return nullptr;
}

mlsdc_status check_op_ptrs(mlsdc_adjoint_t A) {
    for (const Op& o : A->ops) {
        const int np = o.k == OpK::Node ? 6 : o.k == OpK::Fas ? 10 : o.k == OpK::Interp ? 9
                                                                    : o.k == OpK::SolveCoefs ? 0 : 2;
        for (int i = 0; i < np; ++i)
            if (o.p[i] && !adj_of(A, o.p[i])) {
                set_error_text("mlsdc_adjoint: an operand has no adjoint buffer");
                return MLSDC_ERR_INVALID;
            }
    }
    return MLSDC_OK;
}

// the reverse walk of one step whose F_E inputs are in `tape`
mlsdc_status reverse_step(mlsdc_adjoint_t A, const double2* tape, cudaStream_t st, int64_t* launches) {
    mlsdc_t ml = A->ml;
    sdc_level_t F = ml->f, C = ml->c;
    const int ncf = F->plan->nc, ncc = C->plan->nc;
    const int nfn = F->n, ncn = C->n;
    const dim3 gt(grid_for(3 * ncc));
    int64_t n = 0;
    MLSDC_CUDA(cudaMemsetAsync(A->slab, 0, A->slab_n * sizeof(double2), st));
    FasArgs fa;
    std::memset(&fa, 0, sizeof(fa));
    fa.nfn = nfn;
    fa.ncn = ncn;
    for (int i = 0; i < nfn * nfn; ++i) fa.Qf[i] = F->Q[i];
    for (int i = 0; i < ncn * ncn; ++i) fa.Qc[i] = C->Q[i];
    for (int i = 0; i < ncn * nfn; ++i) fa.Pcf[i] = ml->Pcf.a[i];
    for (auto it = A->ops.rbegin(); it != A->ops.rend(); ++it) {
        const Op& o = *it;
        sdc_level_t L = o.L;
        switch (o.k) {
            case OpK::Copy2D:
            case OpK::PadAdd:
                return invalid_arg("mlsdc_adjoint: the operation list holds a time-parallel operation");
            case OpK::CopyLast:
            case OpK::Copy: {
                const size_t cnt = o.k == OpK::Copy ? o.bytes / sizeof(double2) : L->node();
                k_acc_clear<<<grid_for((int)cnt), 256, 0, st>>>(adj_of(A, o.p[0]), adj_of(A, o.p[1]), cnt);
                MLSDC_LAUNCHED("k_acc_clear");
                break;
            }
            case OpK::Bcast:
                k_bcast_ad<<<grid_for(o.n3), 256, 0, st>>>(adj_of(A, o.p[0]), adj_of(A, o.p[1]), o.n3, o.count);
                MLSDC_LAUNCHED("k_bcast_ad");
                break;
            case OpK::FI:
                for (int k = 0; k < std::max(1, o.nodes); ++k) {
                    const size_t sh = (size_t)k * L->node();
                    k_fi_ad<<<grid_for(L->plan->nc), 256, 0, st>>>(adj_of(A, o.p[0]) + sh, adj_of(A, o.p[1]) + sh,
                                                                  L->plan->d_ndeg, L->plan->nc, phys_of(L->prm));
                    MLSDC_LAUNCHED("k_fi_ad");
                    n++;
                }
                n--;  // counted below with the others
                break;
            case OpK::FE:
                // one transpose per node of a node-batched evaluation
                for (int k = 0; k < std::max(1, o.nodes); ++k) {
                    const size_t sh = (size_t)k * L->node();
                    mlsdc_status s = fe_adjoint(L->plan, &L->prm, tape + o.tape_off + sh, adj_of(A, o.p[1]) + sh,
                                                adj_of(A, o.p[0]) + sh, st, &n);
                    if (s != MLSDC_OK) return s;
                }
                n--;  // counted below with the others
                break;
            case OpK::Node:
                k_node_ad<<<grid_for(L->plan->nc), 256, 0, st>>>(adj_of(A, o.p[0]), adj_of(A, o.p[1]),
                                                                adj_of(A, o.p[2]), adj_of(A, o.p[3]),
                                                                adj_of(A, o.p[4]), adj_of(A, o.p[5]), L->plan->d_ndeg,
                                                                recips_of(L, o.dt) + (size_t)o.row.m * (L->plan->R + 1),
                                                                L->plan->nc, o.dt, o.row, phys_of(L->prm));
                MLSDC_LAUNCHED("k_node_ad");
                break;
            case OpK::SolveCoefs:
                // constant coefficients of the step, recomputed by its forward ops: nothing to transpose
                n--;
                break;
            case OpK::Restrict:
                k_restrict_ad<<<gt, 256, 0, st>>>(adj_of(A, o.p[0]), adj_of(A, o.p[1]), ml->d_c2f, ncf, ncc, nfn, o.i0,
                                                 o.i1, ml->Pcf);
                MLSDC_LAUNCHED("k_restrict_ad");
                break;
            case OpK::Fas:
                k_fas_ad<<<gt, 256, 0, st>>>(adj_of(A, o.p[0]), adj_of(A, o.p[1]), adj_of(A, o.p[2]),
                                            adj_of(A, o.p[3]), adj_of(A, o.p[4]), adj_of(A, o.p[5]),
                                            adj_of(A, o.p[6]), adj_of(A, o.p[7]), adj_of(A, o.p[8]),
                                            adj_of(A, o.p[9]), ml->d_c2f, ncf, ncc, o.dt, fa);
                MLSDC_LAUNCHED("k_fas_ad");
                break;
            case OpK::Interp:
                k_interp_ad<<<gt, 256, 0, st>>>(adj_of(A, o.p[0]), adj_of(A, o.p[1]), adj_of(A, o.p[2]),
                                               adj_of(A, o.p[3]), adj_of(A, o.p[4]), adj_of(A, o.p[5]),
                                               adj_of(A, o.p[6]), adj_of(A, o.p[7]), adj_of(A, o.p[8]), ml->d_c2f,
                                               ncf, ncc, nfn, ncn, ml->Pfc);
                MLSDC_LAUNCHED("k_interp_ad");
                break;
        }
        n++;
    }
    if (launches) *launches = n;
    return MLSDC_OK;
}

template <class Enqueue>
mlsdc_status capture_graph(cudaStream_t cap, cudaGraphExec_t* out, Enqueue enqueue) {
    MLSDC_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    mlsdc_status s = enqueue(cap);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(cap, &g);
    if (s != MLSDC_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
    }
    if (e != cudaSuccess) {
        set_error("cudaStreamEndCapture", e);
        return MLSDC_ERR_CUDA;
    }
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        set_error("cudaGraphInstantiate", e);
        return MLSDC_ERR_CUDA;
    }
    return MLSDC_OK;
}

// the operations of one forward step on `work` (tape slot k, or no tape)
mlsdc_status fwd_step(mlsdc_adjoint_t A, int k, int use_graph, cudaStream_t st) {
    double2* tape = k < 0 ? nullptr : A->tape + (size_t)k * A->tape_step;
    if (!use_graph) return run_ops(A->ml, A->ops, st, &A->launches_fwd, tape);
    cudaGraphExec_t* g = k < 0 ? &A->g_fwd : &A->g_tape[k];
    if (!*g) {
        mlsdc_status s = capture_graph(A->cap, g, [&](cudaStream_t cs) {
            return run_ops(A->ml, A->ops, cs, &A->launches_fwd, tape);
        });
        if (s != MLSDC_OK) return s;
    }
    MLSDC_CUDA(cudaGraphLaunch(*g, st));
    return MLSDC_OK;
}

mlsdc_status rev_step(mlsdc_adjoint_t A, int k, int use_graph, cudaStream_t st) {
    const double2* tape = A->tape + (size_t)k * A->tape_step;
    if (!use_graph) return reverse_step(A, tape, st, &A->launches_rev);
    if (!A->g_rev[k]) {
        mlsdc_status s = capture_graph(A->cap, &A->g_rev[k], [&](cudaStream_t cs) {
            return reverse_step(A, tape, cs, &A->launches_rev);
        });
        if (s != MLSDC_OK) return s;
    }
    MLSDC_CUDA(cudaGraphLaunch(A->g_rev[k], st));
    return MLSDC_OK;
}

}  // namespace

extern "C" mlsdc_status mlsdc_adjoint_create(mlsdc_t ml, int n_steps, int checkpoint_every, double dt, int n_iter,
                                             int n_coarse_sweeps, mlsdc_adjoint_t* out) {
    if (!ml || !out || n_steps < 1 || checkpoint_every < 1 || n_iter < 0 || n_coarse_sweeps < 0 || !(dt > 0.0))
        return MLSDC_ERR_INVALID;
    sdc_level_t F = ml->f, C = ml->c;
    if (F->members != 1 || F->plan->precision != MLSDC_FP64 || C->plan->precision != MLSDC_FP64) {
        set_error_text("mlsdc_adjoint_create: needs one member and float64 plans");
        return MLSDC_ERR_INVALID;
    }
    if (F->options || C->options) {
        set_error_text("mlsdc_adjoint_create: the implicit-Coriolis splitting has no adjoint");
        return MLSDC_ERR_INVALID;
    }
    mlsdc_adjoint_t A = new mlsdc_adjoint_s();
    A->ml = ml;
    A->n_steps = n_steps;
    A->every = std::min(checkpoint_every, n_steps);
    A->n_iter = n_iter;
    A->n_c = n_coarse_sweeps;
    A->dt = dt;
    const size_t n3f = F->node();
    const int n_ck = (n_steps + A->every - 1) / A->every;
    bool ok = cudaMalloc((void**)&A->work, n3f * sizeof(double2)) == cudaSuccess &&
              cudaMalloc((void**)&A->lam, n3f * sizeof(double2)) == cudaSuccess &&
              cudaMalloc((void**)&A->ck, (size_t)n_ck * n3f * sizeof(double2)) == cudaSuccess &&
              cudaStreamCreateWithFlags(&A->cap, cudaStreamNonBlocking) == cudaSuccess;
    if (ok) {
        const int fcur = F->cur, ccur = C->cur;
        F->cur = C->cur = 0;
        A->tape_step = build_mlsdc_ops(ml, A->work, dt, n_iter, n_coarse_sweeps, A->ops);
        F->cur = fcur;
        C->cur = ccur;
        ok = cudaMalloc((void**)&A->tape, (size_t)A->every * A->tape_step * sizeof(double2)) == cudaSuccess;
    }
    if (ok) {
        // adjoint buffers mirroring every forward buffer of the step
        std::vector<std::pair<const double2*, size_t>> fw;
        const size_t nf = F->ms(), ncs = C->ms();
        for (sdc_level_t L : {F, C}) {
            const size_t n = L == F ? nf : ncs;
            fw.push_back({L->Th, n});
            for (int b = 0; b < 2; ++b) {
                fw.push_back({L->FI[b], n});
                fw.push_back({L->FE[b], n});
            }
        }
        for (const double2* p : {ml->Ts, ml->FIs, ml->FEs, ml->tau}) fw.push_back({p, ncs});
        A->slab_n = 0;
        for (auto& r : fw) A->slab_n += r.second;
        ok = cudaMalloc((void**)&A->slab, A->slab_n * sizeof(double2)) == cudaSuccess;
        size_t off = 0;
        for (auto& r : fw) {
            A->regions.push_back({r.first, r.second, A->slab + off});
            off += r.second;
        }
        A->regions.push_back({A->work, n3f, A->lam});
    }
    if (!ok) {
        set_error("mlsdc_adjoint_create", cudaGetLastError());
        mlsdc_adjoint_destroy(A);
        return MLSDC_ERR_ALLOC;
    }
    mlsdc_status s = check_op_ptrs(A);
    if (s == MLSDC_OK) s = fe_adjoint_prepare(F->plan);
    if (s == MLSDC_OK) s = fe_adjoint_prepare(C->plan);
    if (s != MLSDC_OK) {
        mlsdc_adjoint_destroy(A);
        return s;
    }
    A->g_tape.assign(A->every, nullptr);
    A->g_rev.assign(A->every, nullptr);
    *out = A;
    return MLSDC_OK;
}

extern "C" mlsdc_status mlsdc_adjoint_destroy(mlsdc_adjoint_t A) {
    if (!A) return MLSDC_ERR_INVALID;
    if (A->g_fwd) cudaGraphExecDestroy(A->g_fwd);
    for (auto g : A->g_tape)
        if (g) cudaGraphExecDestroy(g);
    for (auto g : A->g_rev)
        if (g) cudaGraphExecDestroy(g);
    cudaFree(A->ck);
    cudaFree(A->tape);
    cudaFree(A->work);
    cudaFree(A->lam);
    cudaFree(A->slab);
    if (A->cap) cudaStreamDestroy(A->cap);
    delete A;
    return MLSDC_OK;
}

extern "C" mlsdc_status mlsdc_adjoint_forward(mlsdc_adjoint_t A, const double* state0, double* state_T, int use_graph,
                                              void* stream) {
    if (!A || !state0 || !state_T) return MLSDC_ERR_INVALID;
    MLSDC_ALIGNED("mlsdc_adjoint_forward", {"state0", state0}, {"state_T", state_T});
    cudaStream_t st = (cudaStream_t)stream;
    for (sdc_level_t L : {A->ml->f, A->ml->c}) {  // per-dt tables, before any capture
        mlsdc_status r = prepare_level_tables(L, A->dt, st);
        if (r != MLSDC_OK) return r;
    }
    const size_t bytes = A->ml->f->node() * sizeof(double2);
    MLSDC_CUDA(cudaMemcpyAsync(A->work, state0, bytes, cudaMemcpyDeviceToDevice, st));
    for (int s = 0; s < A->n_steps; ++s) {
        if (s % A->every == 0)
            MLSDC_CUDA(cudaMemcpyAsync(A->ck + (size_t)(s / A->every) * A->ml->f->node(), A->work, bytes,
                                       cudaMemcpyDeviceToDevice, st));
        mlsdc_status r = fwd_step(A, -1, use_graph, st);
        if (r != MLSDC_OK) return r;
    }
    MLSDC_CUDA(cudaMemcpyAsync(state_T, A->work, bytes, cudaMemcpyDeviceToDevice, st));
    A->have_forward = true;
    return MLSDC_OK;
}

extern "C" mlsdc_status mlsdc_adjoint_backward(mlsdc_adjoint_t A, const double* lambda_T, double* lambda_0,
                                               int use_graph, void* stream) {
    if (!A || !lambda_T || !lambda_0) return MLSDC_ERR_INVALID;
    MLSDC_ALIGNED("mlsdc_adjoint_backward", {"lambda_T", lambda_T}, {"lambda_0", lambda_0});
    if (!A->have_forward) {
        set_error_text("mlsdc_adjoint_backward: no forward run has stored the checkpoints");
        return MLSDC_ERR_INVALID;
    }
    cudaStream_t st = (cudaStream_t)stream;
    sdc_level_t F = A->ml->f;
    const size_t n3 = F->node(), bytes = n3 * sizeof(double2);
    const int R = F->plan->R, nc = F->plan->nc;
    MLSDC_CUDA(cudaMemcpyAsync(A->lam, lambda_T, bytes, cudaMemcpyDeviceToDevice, st));
    k_zero_m0_imag<<<1, 256, 0, st>>>(A->lam, R, nc, 3);
    MLSDC_LAUNCHED("k_zero_m0_imag");
    const int n_ck = (A->n_steps + A->every - 1) / A->every;
    for (int seg = n_ck - 1; seg >= 0; --seg) {
        const int s0 = seg * A->every;
        const int len = std::min(A->every, A->n_steps - s0);
        // recompute the segment from its checkpoint, recording every step's F_E inputs
        MLSDC_CUDA(cudaMemcpyAsync(A->work, A->ck + (size_t)seg * n3, bytes, cudaMemcpyDeviceToDevice, st));
        for (int k = 0; k < len; ++k) {
            mlsdc_status r = fwd_step(A, k, use_graph, st);
            if (r != MLSDC_OK) return r;
        }
        for (int k = len - 1; k >= 0; --k) {
            mlsdc_status r = rev_step(A, k, use_graph, st);
            if (r != MLSDC_OK) return r;
        }
    }
    k_zero_m0_imag<<<1, 256, 0, st>>>(A->lam, R, nc, 3);
    MLSDC_LAUNCHED("k_zero_m0_imag");
    MLSDC_CUDA(cudaMemcpyAsync(lambda_0, A->lam, bytes, cudaMemcpyDeviceToDevice, st));
    return MLSDC_OK;
}

extern "C" mlsdc_status mlsdc_adjoint_launch_count(mlsdc_adjoint_t A, int64_t* forward_step, int64_t* reverse_step) {
    if (!A) return MLSDC_ERR_INVALID;
    if (forward_step) *forward_step = A->launches_fwd;
    if (reverse_step) *reverse_step = A->launches_rev;
    return MLSDC_OK;
}

extern "C" mlsdc_status swe_explicit_rhs_adjoint(sh_plan_t p, const swe_params* prm, const double* state,
                                                 double* lambda, double* state_bar, void* stream) {
    if (!p || !prm || !state || !lambda || !state_bar) return MLSDC_ERR_INVALID;
    MLSDC_ALIGNED("swe_explicit_rhs_adjoint", {"state", state}, {"lambda", lambda}, {"state_bar", state_bar});
    if (p->precision != MLSDC_FP64 || state_bar == lambda || state_bar == state || lambda == state)
        return MLSDC_ERR_INVALID;
    mlsdc_status s = fe_adjoint_prepare(p);
    if (s != MLSDC_OK) return s;
    return fe_adjoint(p, prm, (const double2*)state, (double2*)lambda, (double2*)state_bar, (cudaStream_t)stream,
                      nullptr);
}

extern "C" mlsdc_status mlsdc_profile_rhs_adjoint(sh_plan_t p, const swe_params* prm, const double* state,
                                                  double* lambda, double* state_bar, int reps, float* ms_host,
                                                  void* stream) {
    if (!p || !prm || !state || !lambda || !state_bar || reps < 1 || !ms_host) return MLSDC_ERR_INVALID;
    MLSDC_ALIGNED("mlsdc_profile_rhs_adjoint", {"state", state}, {"lambda", lambda}, {"state_bar", state_bar});
    if (p->precision != MLSDC_FP64 || state_bar == lambda || state_bar == state || lambda == state)
        return MLSDC_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    mlsdc_status s = fe_adjoint_prepare(p);
    if (s != MLSDC_OK) return s;
    const int R = p->R;
    const size_t ss = synth_ad_smem(R), gs = grid_ad_smem(p->I);
    const double2* x = (const double2*)state;
    double2* lam = (double2*)lambda;
    double2* xb = (double2*)state_bar;
    auto stage = [&](int k, cudaStream_t cs) -> mlsdc_status {
        if (k == 0)
            k_synth_ad<<<p->n_synth, 32 * kAdSynthWarps, ss, cs>>>(x, lam, p->d_P, p->d_H, p->d_invnn, p->d_synth, R,
                                                                  p->J2, p->nc, prm->a, 1.0 / prm->a, p->d_four_in);
        else if (k == 1)
            k_grid_ad<<<p->J, 256, gs, cs>>>(p->d_four_in, p->d_four_out, p->d_lat, p->d_tw, R, p->I, p->logI, p->J,
                                             2.0 * prm->omega);
        else
            k_anal_ad<<<p->n_anal, 32 * anal_warps(p->J2), 0, cs>>>(p->d_four_out, p->d_P, p->d_H, p->d_invnn,
                                                                   p->d_anal, R, p->J2, p->nc, prm->a, 1.0 / prm->a,
                                                                   xb, lam);
        MLSDC_LAUNCHED("profile_rhs_adjoint");
        return MLSDC_OK;
    };
    // one full evaluation first so every stage reads valid inputs
    if ((s = fe_adjoint(p, prm, x, lam, xb, st, nullptr)) != MLSDC_OK) return s;
    for (int k = 0; k < 3 && s == MLSDC_OK; ++k)
        s = time_in_graph(st, reps, &ms_host[k], [&](cudaStream_t cs) { return stage(k, cs); });
    return s;
}

extern "C" mlsdc_status mlsdc_phi_misfit(sh_plan_t p, const double* state, const double* phi_target, double* J,
                                         double* lambda, void* stream) {
    if (!p || !state || !phi_target || !J || !lambda) return MLSDC_ERR_INVALID;
    MLSDC_ALIGNED("mlsdc_phi_misfit", {"state", state}, {"phi_target", phi_target}, {"lambda", lambda});
    k_misfit<<<1, 1024, 0, (cudaStream_t)stream>>>((const double2*)state, (const double2*)phi_target, p->R, p->nc, J,
                                                   (double2*)lambda);
    MLSDC_LAUNCHED("k_misfit");
    return MLSDC_OK;
}
