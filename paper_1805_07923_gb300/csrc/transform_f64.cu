// Float64 spherical-harmonic transforms and the explicit shallow-water
// right-hand side (Sec. 3, Eqs. spectral_to_physical_space,
// fourier_transform, legendre_transform; Sec. 2 and Sec. 4.1 for F_E).
//
// Data flow of one F_E evaluation (three launches):
//   k_synth_rhs_f64   per (m, 32 latitudes): Legendre sums over n, split in
//                     even/odd n - m so one pass serves a northern latitude
//                     and its southern mirror (P^m_n(-mu) = (-1)^(n-m) P^m_n(mu),
//                     H^m_n(-mu) = -(-1)^(n-m) H^m_n(mu)); writes the Fourier
//                     coefficients of zeta, Phi', U, V   -> four_in[4][J][R+1]
//   k_grid_rhs_f64    per latitude: two packed complex inverse FFTs (two real
//                     fields each), the grid products A..E, three packed
//                     forward FFTs, weights w/(1-mu^2)/I (E: w/I)
//                                                      -> four_out[5][J][R+1]
//   k_anal_rhs_f64    per (m, 32 degrees): Gaussian quadrature sums over the
//                     northern latitudes with even/odd combinations, then
//                     F_E = [-div(C,D), -div(A,B), curl(A,B) + n(n+1)/a^2 E].
// The grid fields never leave shared memory.
#include <cmath>

#include "internal.h"

namespace mlsdc {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ void cfma(double2& acc, double p, double2 c) {
    acc.x = fma(p, c.x, acc.x);
    acc.y = fma(p, c.y, acc.y);
}
// i * m * z
__device__ __forceinline__ double2 cim(double m, double2 z) { return make_double2(-m * z.y, m * z.x); }

__device__ __forceinline__ int bitrev(int k, int logI) { return (int)(__brev((unsigned)k) >> (32 - logI)); }

// In-place radix-2 decimation-in-time FFT of `narr` complex arrays of length
// Hn = I/2 that sit back to back in shared memory, input in bit-reversed
// order, output in natural order.  Forward: sum_k z_k exp(-2 pi i j k / Hn);
// inverse uses conjugate twiddles (no normalisation).  tw[k] = exp(-2 pi i k / I)
// for k < I/2, so the length-Hn twiddles are tw[2 k].
__device__ void fft_dit_f64(double2* x, int narr, int Hn, int logH, const double2* __restrict__ tw,
                            bool inverse) {
    const int half = Hn >> 1;
    for (int s = 0; s < logH; ++s) {
        const int h = 1 << s;
        const int tstride = (half >> s) * 2;
        for (int t = threadIdx.x; t < narr * half; t += blockDim.x) {
            const int a = t / half;
            const int b = t - a * half;
            const int pos = b & (h - 1);
            const int i0 = ((b >> s) << (s + 1)) + pos;
            double2 w = __ldg(&tw[pos * tstride]);
            if (inverse) w.y = -w.y;
            double2* xa = x + a * Hn;
            const double2 u = xa[i0];
            const double2 v = cmul(xa[i0 + h], w);
            xa[i0] = cadd(u, v);
            xa[i0 + h] = csub(u, v);
        }
        __syncthreads();
    }
}

// Real DFTs of length I through complex DFTs of length I/2 over the packed
// samples z_k = x_{2k} + i x_{2k+1} of ONE real row (packing two different
// fields would tie the smaller field's rounding error to the larger one).
// Stored coefficients F[0..R] (R < I/2) of a real row; Im F_0 is ignored.
__device__ __forceinline__ double2 coef(const double2* __restrict__ F, int m, int R) {
    if (m == 0) return make_double2(F[0].x, 0.0);
    if (m <= R) return F[m];
    return make_double2(0.0, 0.0);
}

// Packed spectrum Z_k (k < I/2) whose unnormalised inverse DFT of length I/2
// is z_k = x_{2k} + i x_{2k+1}, x_n = sum_m X_m e^{2 pi i m n / I} (X Hermitian):
// Z_k = (X_k + conj X_{I/2-k}) + i (X_k - conj X_{I/2-k}) e^{+2 pi i k / I}.
__device__ __forceinline__ double2 irfft_pack(const double2* __restrict__ F, int k, int R, int Hn,
                                              const double2* __restrict__ tw) {
    const double2 a = coef(F, k, R);
    double2 c = coef(F, Hn - k, R);
    c.y = -c.y;
    const double2 s = cadd(a, c);
    double2 w = __ldg(&tw[k]);
    w.y = -w.y;
    const double2 d = cmul(csub(a, c), w);
    return make_double2(s.x - d.y, s.y + d.x);
}

// X_m = E_m + e^{-2 pi i m / I} O_m from the forward DFT Z of the packed row,
// E_m = (Z_m + conj Z_{I/2-m}) / 2, O_m = (Z_m - conj Z_{I/2-m}) / (2 i).
__device__ __forceinline__ double2 rfft_unpack(const double2* z, int m, int Hn, const double2* __restrict__ tw) {
    const double2 Z = z[m];
    double2 Zc = z[(Hn - m) & (Hn - 1)];
    Zc.y = -Zc.y;
    const double2 E = make_double2(0.5 * (Z.x + Zc.x), 0.5 * (Z.y + Zc.y));
    const double2 dz = csub(Z, Zc);
    const double2 O = make_double2(0.5 * dz.y, -0.5 * dz.x);
    return cadd(E, cmul(__ldg(&tw[m]), O));
}

// ---------------------------------------------------------------------------
// F_E synthesis: Fourier coefficients of zeta, Phi', U, V at every latitude.
// U^m = (1/a) sum_n [ i m chi P - psi H ],  V^m = (1/a) sum_n [ i m psi P + chi H ]
// with psi, chi = -a^2/(n(n+1)) (zeta, delta) (Helmholtz, Sec. 2).
__global__ void __launch_bounds__(32) k_synth_rhs_f64(const double2* __restrict__ state,
                                                      const double* __restrict__ P,
                                                      const double* __restrict__ H,
                                                      const Chunk* __restrict__ chunks, int R, int J2,
                                                      int nc, double a, double2* __restrict__ four) {
    extern __shared__ double2 sc[];  // [nm][4]: zeta, Phi', chi, psi
    const Chunk ch = chunks[blockIdx.x];
    const int m = ch.m;
    const int nm = R + 1 - m;
    const int off = m * (R + 1) - m * (m - 1) / 2;
    for (int k = threadIdx.x; k < nm; k += blockDim.x) {
        const int n = m + k;
        const double s = n > 0 ? -a * a / (n * (n + 1.0)) : 0.0;
        const double2 ph = state[off + k];
        const double2 ze = state[nc + off + k];
        const double2 de = state[2 * nc + off + k];
        sc[4 * k + 0] = ze;
        sc[4 * k + 1] = ph;
        sc[4 * k + 2] = cscale(de, s);
        sc[4 * k + 3] = cscale(ze, s);
    }
    __syncthreads();
    const int j = ch.start + threadIdx.x;
    if (j >= J2) return;
    double2 ez{0, 0}, ep{0, 0}, exP{0, 0}, esP{0, 0}, esH{0, 0}, exH{0, 0};
    double2 oz{0, 0}, op{0, 0}, oxP{0, 0}, osP{0, 0}, osH{0, 0}, oxH{0, 0};
    const double* Pm = P + (size_t)off * J2 + j;
    const double* Hm = H + (size_t)off * J2 + j;
    int k = 0;
    for (; k + 1 < nm; k += 2) {
        const double p0 = Pm[(size_t)k * J2], h0 = Hm[(size_t)k * J2];
        const double p1 = Pm[(size_t)(k + 1) * J2], h1 = Hm[(size_t)(k + 1) * J2];
        const double2 z0 = sc[4 * k], f0 = sc[4 * k + 1], x0 = sc[4 * k + 2], s0 = sc[4 * k + 3];
        const double2 z1 = sc[4 * k + 4], f1 = sc[4 * k + 5], x1 = sc[4 * k + 6], s1 = sc[4 * k + 7];
        cfma(ez, p0, z0); cfma(ep, p0, f0); cfma(exP, p0, x0); cfma(esP, p0, s0);
        cfma(esH, h0, s0); cfma(exH, h0, x0);
        cfma(oz, p1, z1); cfma(op, p1, f1); cfma(oxP, p1, x1); cfma(osP, p1, s1);
        cfma(osH, h1, s1); cfma(oxH, h1, x1);
    }
    if (k < nm) {
        const double p0 = Pm[(size_t)k * J2], h0 = Hm[(size_t)k * J2];
        const double2 z0 = sc[4 * k], f0 = sc[4 * k + 1], x0 = sc[4 * k + 2], s0 = sc[4 * k + 3];
        cfma(ez, p0, z0); cfma(ep, p0, f0); cfma(exP, p0, x0); cfma(esP, p0, s0);
        cfma(esH, h0, s0); cfma(exH, h0, x0);
    }
    const double ia = 1.0 / a;
    const double dm = (double)m;
    const int J = 2 * J2;
    const int jS = J - 1 - j;
    const size_t fs = (size_t)J * (R + 1);
    // north: P-sums e + o, H-sums e + o; south: P-sums e - o, H-sums o - e
    const double2 zN = cadd(ez, oz), zS = csub(ez, oz);
    const double2 pN = cadd(ep, op), pS = csub(ep, op);
    const double2 xPN = cadd(exP, oxP), xPS = csub(exP, oxP);
    const double2 sPN = cadd(esP, osP), sPS = csub(esP, osP);
    const double2 sHN = cadd(esH, osH), sHS = csub(osH, esH);
    const double2 xHN = cadd(exH, oxH), xHS = csub(oxH, exH);
    four[0 * fs + (size_t)j * (R + 1) + m] = zN;
    four[0 * fs + (size_t)jS * (R + 1) + m] = zS;
    four[1 * fs + (size_t)j * (R + 1) + m] = pN;
    four[1 * fs + (size_t)jS * (R + 1) + m] = pS;
    four[2 * fs + (size_t)j * (R + 1) + m] = cscale(csub(cim(dm, xPN), sHN), ia);
    four[2 * fs + (size_t)jS * (R + 1) + m] = cscale(csub(cim(dm, xPS), sHS), ia);
    four[3 * fs + (size_t)j * (R + 1) + m] = cscale(cadd(cim(dm, sPN), xHN), ia);
    four[3 * fs + (size_t)jS * (R + 1) + m] = cscale(cadd(cim(dm, sPS), xHS), ia);
}

// ---------------------------------------------------------------------------
// Per latitude: grid values of zeta, Phi', U, V by inverse DFT, the products
// A = (zeta+f)U, B = (zeta+f)V, C = Phi'U, D = Phi'V, E = (U^2+V^2)/(2(1-mu^2)),
// and their forward DFTs for m <= R scaled by w/(1-mu^2)/I (A..D) or w/I (E).
__global__ void __launch_bounds__(256) k_grid_rhs_f64(const double2* __restrict__ four_in,
                                                      double2* __restrict__ four_out,
                                                      const double* __restrict__ mu,
                                                      const double* __restrict__ w,
                                                      const double2* __restrict__ tw, int R, int I,
                                                      int logI, int J, double two_omega) {
    extern __shared__ double2 sx[];  // [9][I/2]: zeta, Phi', U, V packed rows, then A..E
    const int j = blockIdx.x;
    const int Hn = I >> 1, logH = logI - 1;
    const size_t fs = (size_t)J * (R + 1);
    for (int t = threadIdx.x; t < 4 * Hn; t += blockDim.x) {
        const int f = t / Hn, k = t - f * Hn;
        sx[f * Hn + bitrev(k, logH)] = irfft_pack(four_in + f * fs + (size_t)j * (R + 1), k, R, Hn, tw);
    }
    __syncthreads();
    fft_dit_f64(sx, 4, Hn, logH, tw, true);
    const double muj = mu[j];
    const double f = two_omega * muj;
    const double rc = 1.0 / (1.0 - muj * muj);
    double2* y = sx + 4 * Hn;
    for (int k = threadIdx.x; k < Hn; k += blockDim.x) {
        // .x holds longitude 2k, .y longitude 2k+1
        const double2 z = sx[k], p = sx[Hn + k], u = sx[2 * Hn + k], v = sx[3 * Hn + k];
        const double zf0 = z.x + f, zf1 = z.y + f;
        const int r = bitrev(k, logH);
        y[r] = make_double2(zf0 * u.x, zf1 * u.y);                                   // A
        y[Hn + r] = make_double2(zf0 * v.x, zf1 * v.y);                              // B
        y[2 * Hn + r] = make_double2(p.x * u.x, p.y * u.y);                          // C
        y[3 * Hn + r] = make_double2(p.x * v.x, p.y * v.y);                          // D
        y[4 * Hn + r] = make_double2(0.5 * (u.x * u.x + v.x * v.x) * rc,             // E
                                     0.5 * (u.y * u.y + v.y * v.y) * rc);
    }
    __syncthreads();
    fft_dit_f64(y, 5, Hn, logH, tw, false);
    const double sAD = w[j] * rc / I;
    const double sE = w[j] / I;
    for (int t = threadIdx.x; t < 5 * (R + 1); t += blockDim.x) {
        const int fld = t / (R + 1);
        const int m = t - fld * (R + 1);
        const double2 X = rfft_unpack(y + fld * Hn, m, Hn, tw);
        four_out[(size_t)fld * fs + (size_t)j * (R + 1) + m] = cscale(X, fld < 4 ? sAD : sE);
    }
}

// ---------------------------------------------------------------------------
// F_E analysis (integration by parts of the mu-derivatives, Sec. 2 operators):
// div(X,Y)^m_n = (1/a) sum_j [ i m X' P - Y' H ], curl(X,Y)^m_n = (1/a) sum_j [ i m Y' P + X' H ]
// with X', Y' the weighted Fourier coefficients; E^m_n = sum_j E' P.
__global__ void __launch_bounds__(32) k_anal_rhs_f64(const double2* __restrict__ four_out,
                                                     const double* __restrict__ P,
                                                     const double* __restrict__ H,
                                                     const Chunk* __restrict__ chunks, int R, int J2,
                                                     int nc, double a, double2* __restrict__ FE) {
    __shared__ double2 sG[32][5][2];  // [lat][field A..E][even, odd]
    __shared__ double sP[32][33];
    __shared__ double sH[32][33];
    const Chunk ch = chunks[blockIdx.x];
    const int m = ch.m;
    const int nm = R + 1 - m;
    const int off = m * (R + 1) - m * (m - 1) / 2;
    const int k0 = ch.start;
    const int lane = threadIdx.x;
    const int k = k0 + lane;
    const int par = k & 1;
    const int J = 2 * J2;
    const size_t fs = (size_t)J * (R + 1);
    const int rows = min(32, nm - k0);
    double2 aC{0, 0}, aA{0, 0}, aB{0, 0}, aE{0, 0}, hD{0, 0}, hB{0, 0}, hA{0, 0};
    for (int jt = 0; jt < J2; jt += 32) {
        const int nl = min(32, J2 - jt);
        for (int t = lane; t < nl * 5; t += 32) {
            const int jj = t / 5, f = t - jj * 5;
            const int jn = jt + jj, js = J - 1 - jn;
            const double2 gN = four_out[(size_t)f * fs + (size_t)jn * (R + 1) + m];
            const double2 gS = four_out[(size_t)f * fs + (size_t)js * (R + 1) + m];
            sG[jj][f][0] = cadd(gN, gS);
            sG[jj][f][1] = csub(gN, gS);
        }
        for (int r = 0; r < rows; ++r) {
            if (lane < nl) {
                sP[r][lane] = P[(size_t)(off + k0 + r) * J2 + jt + lane];
                sH[r][lane] = H[(size_t)(off + k0 + r) * J2 + jt + lane];
            }
        }
        __syncwarp();
        if (lane < rows) {
            for (int jj = 0; jj < nl; ++jj) {
                const double p = sP[lane][jj], h = sH[lane][jj];
                cfma(aC, p, sG[jj][2][par]);
                cfma(aA, p, sG[jj][0][par]);
                cfma(aB, p, sG[jj][1][par]);
                cfma(aE, p, sG[jj][4][par]);
                cfma(hD, h, sG[jj][3][par ^ 1]);
                cfma(hB, h, sG[jj][1][par ^ 1]);
                cfma(hA, h, sG[jj][0][par ^ 1]);
            }
        }
        __syncwarp();
    }
    if (lane >= rows) return;
    const int n = m + k;
    const double ia = 1.0 / a;
    const double dm = (double)m;
    const double2 divCD = cscale(csub(cim(dm, aC), hD), ia);
    const double2 divAB = cscale(csub(cim(dm, aA), hB), ia);
    const double2 curlAB = cscale(cadd(cim(dm, aB), hA), ia);
    const double lap = n * (n + 1.0) * ia * ia;
    double2 f0 = make_double2(-divCD.x, -divCD.y);
    double2 f1 = make_double2(-divAB.x, -divAB.y);
    double2 f2 = make_double2(curlAB.x + lap * aE.x, curlAB.y + lap * aE.y);
    if (m == 0) f0.y = f1.y = f2.y = 0.0;
    FE[off + k] = f0;
    FE[nc + off + k] = f1;
    FE[2 * nc + off + k] = f2;
}

// ---------------------------------------------------------------------------
// Scalar transforms (sh_inverse / sh_forward).
__global__ void __launch_bounds__(32) k_synth_scalar_f64(const double2* __restrict__ spec,
                                                         const double* __restrict__ P,
                                                         const Chunk* __restrict__ chunks, int R,
                                                         int J2, int nc, double2* __restrict__ four) {
    extern __shared__ double2 sc[];
    const int fld = blockIdx.y;
    const Chunk ch = chunks[blockIdx.x];
    const int m = ch.m;
    const int nm = R + 1 - m;
    const int off = m * (R + 1) - m * (m - 1) / 2;
    for (int k = threadIdx.x; k < nm; k += blockDim.x) sc[k] = spec[(size_t)fld * nc + off + k];
    __syncthreads();
    const int j = ch.start + threadIdx.x;
    if (j >= J2) return;
    double2 e{0, 0}, o{0, 0};
    const double* Pm = P + (size_t)off * J2 + j;
    int k = 0;
    for (; k + 1 < nm; k += 2) {
        cfma(e, Pm[(size_t)k * J2], sc[k]);
        cfma(o, Pm[(size_t)(k + 1) * J2], sc[k + 1]);
    }
    if (k < nm) cfma(e, Pm[(size_t)k * J2], sc[k]);
    const int J = 2 * J2;
    const size_t base = (size_t)fld * J * (R + 1);
    four[base + (size_t)j * (R + 1) + m] = cadd(e, o);
    four[base + (size_t)(J - 1 - j) * (R + 1) + m] = csub(e, o);
}

// Inverse real DFT of one row per block: coefficients m <= R -> I grid values.
__global__ void __launch_bounds__(128) k_fft_inv_rows_f64(const double2* __restrict__ four,
                                                          double* __restrict__ grid,
                                                          const double2* __restrict__ tw, int R, int I,
                                                          int logI) {
    extern __shared__ double2 sx[];
    const int row = blockIdx.x;
    const int Hn = I >> 1, logH = logI - 1;
    const double2* F = four + (size_t)row * (R + 1);
    for (int k = threadIdx.x; k < Hn; k += blockDim.x) sx[bitrev(k, logH)] = irfft_pack(F, k, R, Hn, tw);
    __syncthreads();
    fft_dit_f64(sx, 1, Hn, logH, tw, true);
    double2* g = (double2*)(grid + (size_t)row * I);
    for (int k = threadIdx.x; k < Hn; k += blockDim.x) g[k] = sx[k];
}

// Forward real DFT of one row per block, coefficients m <= R scaled by w_j / I.
__global__ void __launch_bounds__(128) k_fft_fwd_rows_f64(const double* __restrict__ grid,
                                                          double2* __restrict__ four,
                                                          const double* __restrict__ w,
                                                          const double2* __restrict__ tw, int R, int I,
                                                          int logI, int J) {
    extern __shared__ double2 sx[];
    const int row = blockIdx.x;
    const int Hn = I >> 1, logH = logI - 1;
    const double2* g = (const double2*)(grid + (size_t)row * I);
    for (int k = threadIdx.x; k < Hn; k += blockDim.x) sx[bitrev(k, logH)] = g[k];
    __syncthreads();
    fft_dit_f64(sx, 1, Hn, logH, tw, false);
    const double s = w[row % J] / I;
    for (int m = threadIdx.x; m <= R; m += blockDim.x)
        four[(size_t)row * (R + 1) + m] = cscale(rfft_unpack(sx, m, Hn, tw), s);
}

__global__ void __launch_bounds__(32) k_anal_scalar_f64(const double2* __restrict__ four,
                                                        const double* __restrict__ P,
                                                        const Chunk* __restrict__ chunks, int R, int J2,
                                                        int nc, double2* __restrict__ spec) {
    __shared__ double2 sG[32][2];
    __shared__ double sP[32][33];
    const int fld = blockIdx.y;
    const Chunk ch = chunks[blockIdx.x];
    const int m = ch.m;
    const int nm = R + 1 - m;
    const int off = m * (R + 1) - m * (m - 1) / 2;
    const int k0 = ch.start;
    const int lane = threadIdx.x;
    const int par = (k0 + lane) & 1;
    const int J = 2 * J2;
    const double2* F = four + (size_t)fld * J * (R + 1);
    const int rows = min(32, nm - k0);
    double2 acc{0, 0};
    for (int jt = 0; jt < J2; jt += 32) {
        const int nl = min(32, J2 - jt);
        if (lane < nl) {
            const double2 gN = F[(size_t)(jt + lane) * (R + 1) + m];
            const double2 gS = F[(size_t)(J - 1 - jt - lane) * (R + 1) + m];
            sG[lane][0] = cadd(gN, gS);
            sG[lane][1] = csub(gN, gS);
        }
        for (int r = 0; r < rows; ++r)
            if (lane < nl) sP[r][lane] = P[(size_t)(off + k0 + r) * J2 + jt + lane];
        __syncwarp();
        if (lane < rows)
            for (int jj = 0; jj < nl; ++jj) cfma(acc, sP[lane][jj], sG[jj][par]);
        __syncwarp();
    }
    if (lane >= rows) return;
    if (m == 0) acc.y = 0.0;
    spec[(size_t)fld * nc + off + k0 + lane] = acc;
}

mlsdc_status rhs_explicit_f64(sh_plan_t p, const swe_params* prm, const double* state, double* FE,
                              cudaStream_t st, int64_t* launches, int stage) {
    const int R = p->R;
    if (stage == 0 || stage < 0) {
    size_t smem_syn = sizeof(double2) * 4 * (R + 1);
    k_synth_rhs_f64<<<p->n_synth, 32, smem_syn, st>>>((const double2*)state, p->d_P, p->d_H, p->d_synth,
                                                      R, p->J2, p->nc, prm->a, p->d_four_in);
    MLSDC_LAUNCHED("k_synth_rhs_f64");
    }
    if (stage == 1 || stage < 0) {
    size_t smem_grid = sizeof(double2) * 9 * (p->I / 2);
    k_grid_rhs_f64<<<p->J, 256, smem_grid, st>>>(p->d_four_in, p->d_four_out, p->d_mu, p->d_w, p->d_tw, R,
                                                 p->I, p->logI, p->J, 2.0 * prm->omega);
    MLSDC_LAUNCHED("k_grid_rhs_f64");
    }
    if (stage == 2 || stage < 0) {
    k_anal_rhs_f64<<<p->n_anal, 32, 0, st>>>(p->d_four_out, p->d_P, p->d_H, p->d_anal, R, p->J2, p->nc,
                                             prm->a, (double2*)FE);
    MLSDC_LAUNCHED("k_anal_rhs_f64");
    }
    if (launches) *launches += stage < 0 ? 3 : 1;
    return MLSDC_OK;
}

static mlsdc_status set_smem(const void* fn, size_t bytes) {
    if (bytes > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) {
            set_error("cudaFuncSetAttribute", e);
            return MLSDC_ERR_CUDA;
        }
    }
    return MLSDC_OK;
}

mlsdc_status f64_prepare(sh_plan_t p) {
    mlsdc_status s;
    if ((s = set_smem((const void*)k_grid_rhs_f64, sizeof(double2) * 9 * (p->I / 2))) != MLSDC_OK) return s;
    return MLSDC_OK;
}

}  // namespace mlsdc

using namespace mlsdc;

extern "C" mlsdc_status sh_inverse(sh_plan_t p, const double* spec, double* grid, int nf, void* stream) {
    if (!p || !spec || !grid || nf < 1 || nf > kMaxFields) return MLSDC_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    const int R = p->R;
    dim3 gs(p->n_synth, nf);
    k_synth_scalar_f64<<<gs, 32, sizeof(double2) * (R + 1), st>>>((const double2*)spec, p->d_P, p->d_synth, R,
                                                                  p->J2, p->nc, p->d_four_in);
    MLSDC_LAUNCHED("k_synth_scalar_f64");
    const int rows = nf * p->J;
    k_fft_inv_rows_f64<<<rows, 128, sizeof(double2) * (p->I / 2), st>>>(p->d_four_in, grid, p->d_tw, R, p->I,
                                                                       p->logI);
    MLSDC_LAUNCHED("k_fft_inv_rows_f64");
    return MLSDC_OK;
}

extern "C" mlsdc_status sh_forward(sh_plan_t p, const double* grid, double* spec, int nf, void* stream) {
    if (!p || !spec || !grid || nf < 1 || nf > kMaxFields) return MLSDC_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    const int R = p->R;
    const int rows = nf * p->J;
    k_fft_fwd_rows_f64<<<rows, 128, sizeof(double2) * (p->I / 2), st>>>(grid, p->d_four_out, p->d_w, p->d_tw, R,
                                                                       p->I, p->logI, p->J);
    MLSDC_LAUNCHED("k_fft_fwd_rows_f64");
    dim3 ga(p->n_anal, nf);
    k_anal_scalar_f64<<<ga, 32, 0, st>>>(p->d_four_out, p->d_P, p->d_anal, R, p->J2, p->nc, (double2*)spec);
    MLSDC_LAUNCHED("k_anal_scalar_f64");
    return MLSDC_OK;
}

extern "C" mlsdc_status swe_explicit_rhs(sh_plan_t p, const swe_params* prm, const double* state, double* FE,
                                         void* stream) {
    if (!p || !prm || !state || !FE || state == FE) return MLSDC_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    if (p->precision == MLSDC_FP64) return rhs_explicit_f64(p, prm, state, FE, st, nullptr, -1);
    return rhs_explicit_mp(p, prm, state, FE, st, nullptr, -1);
}

extern "C" mlsdc_status mlsdc_profile_rhs(sh_plan_t p, const swe_params* prm, const double* state, double* FE,
                                          int reps, float* ms_host, void* stream) {
    if (!p || !prm || !state || !FE || state == FE || reps < 1 || !ms_host) return MLSDC_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    mlsdc_status s;
    // one full evaluation first so every stage reads valid inputs
    if (p->precision == MLSDC_FP64) s = rhs_explicit_f64(p, prm, state, FE, st, nullptr, -1);
    else s = rhs_explicit_mp(p, prm, state, FE, st, nullptr, -1);
    if (s != MLSDC_OK) return s;
    cudaEvent_t e0, e1;
    MLSDC_CUDA(cudaEventCreate(&e0));
    MLSDC_CUDA(cudaEventCreate(&e1));
    for (int stage = 0; stage < 3; ++stage) {
        MLSDC_CUDA(cudaEventRecord(e0, st));
        for (int r = 0; r < reps; ++r) {
            if (p->precision == MLSDC_FP64) s = rhs_explicit_f64(p, prm, state, FE, st, nullptr, stage);
            else s = rhs_explicit_mp(p, prm, state, FE, st, nullptr, stage);
            if (s != MLSDC_OK) break;
        }
        MLSDC_CUDA(cudaEventRecord(e1, st));
        MLSDC_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        MLSDC_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        ms_host[stage] = ms / reps;
        if (s != MLSDC_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return s;
}
