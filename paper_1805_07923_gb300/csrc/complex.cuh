// Complex helpers and shared-memory real FFTs, templated on the real type
// (double for the float64 path, float for the mixed-precision path).
#pragma once

#include <cuda_runtime.h>

namespace mlsdc {

template <class T> struct cplx;
template <> struct cplx<double> { using t = double2; };
template <> struct cplx<float> { using t = float2; };
template <class T> using C_t = typename cplx<T>::t;

__device__ __forceinline__ double2 mkc(double x, double y) { return make_double2(x, y); }
__device__ __forceinline__ float2 mkc(float x, float y) { return make_float2(x, y); }

template <class C> __device__ __forceinline__ C cmul(C a, C b) { return mkc(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
template <class C> __device__ __forceinline__ C cadd(C a, C b) { return mkc(a.x + b.x, a.y + b.y); }
template <class C> __device__ __forceinline__ C csub(C a, C b) { return mkc(a.x - b.x, a.y - b.y); }
template <class C, class T> __device__ __forceinline__ C cscale(C a, T s) { return mkc(a.x * s, a.y * s); }
template <class C> __device__ __forceinline__ C cconj(C a) { return mkc(a.x, -a.y); }
__device__ __forceinline__ void cfma(double2& acc, double p, double2 c) {
    acc.x = fma(p, c.x, acc.x);
    acc.y = fma(p, c.y, acc.y);
}
__device__ __forceinline__ void cfma(float2& acc, float p, float2 c) {
    acc.x = fmaf(p, c.x, acc.x);
    acc.y = fmaf(p, c.y, acc.y);
}
// i * m * z
template <class C, class T> __device__ __forceinline__ C cim(T m, C z) { return mkc(-m * z.y, m * z.x); }

__device__ __forceinline__ int bitrev(int k, int logn) { return (int)(__brev((unsigned)k) >> (32 - logn)); }

// In-place radix-2 decimation-in-time FFT of `narr` complex arrays of length
// Hn = I/2 that sit back to back in shared memory, input in bit-reversed
// order, output in natural order.  Forward: sum_k z_k exp(-2 pi i j k / Hn);
// inverse uses conjugate twiddles (no normalisation).  tw[k] = exp(-2 pi i k / I)
// for k < I/2, so the length-Hn twiddles are tw[2 k].
template <class C>
__device__ void fft_dit(C* x, int narr, int Hn, int logH, const C* __restrict__ tw, bool inverse) {
    const int half = Hn >> 1;
    for (int s = 0; s < logH; ++s) {
        const int h = 1 << s;
        const int tstride = (half >> s) * 2;
        for (int t = threadIdx.x; t < narr * half; t += blockDim.x) {
            const int a = t >> (logH - 1);
            const int b = t & (half - 1);
            const int pos = b & (h - 1);
            const int i0 = ((b >> s) << (s + 1)) + pos;
            C w = __ldg(&tw[pos * tstride]);
            if (inverse) w.y = -w.y;
            C* xa = x + a * Hn;
            const C u = xa[i0];
            const C v = cmul(xa[i0 + h], w);
            xa[i0] = cadd(u, v);
            xa[i0 + h] = csub(u, v);
        }
        __syncthreads();
    }
}

// In-place radix-2 decimation-in-frequency FFT, same conventions as fft_dit
// but natural-order input and bit-reversed output.  Pairing it with fft_dit
// (bit-reversed input) lets a pointwise stage run between the two transforms
// in the permuted order, so no permutation is ever written out.
template <class C>
__device__ void fft_dif(C* x, int narr, int Hn, int logH, const C* __restrict__ tw, bool inverse) {
    const int half = Hn >> 1;
    for (int s = logH - 1; s >= 0; --s) {
        const int h = 1 << s;
        const int tstride = (half >> s) * 2;
        for (int t = threadIdx.x; t < narr * half; t += blockDim.x) {
            const int a = t >> (logH - 1);
            const int b = t & (half - 1);
            const int pos = b & (h - 1);
            const int i0 = ((b >> s) << (s + 1)) + pos;
            C w = __ldg(&tw[pos * tstride]);
            if (inverse) w.y = -w.y;
            C* xa = x + a * Hn;
            const C u = xa[i0];
            const C v = xa[i0 + h];
            xa[i0] = cadd(u, v);
            xa[i0 + h] = cmul(csub(u, v), w);
        }
        __syncthreads();
    }
}

// Mixed radix-4 (and one radix-2 stage when log2 N is odd) versions of the
// same pair: fft4_dif takes natural-order input to an output in the
// base-4 digit-reversed order of its stages, fft4_dit takes that order back
// to natural order, so the two compose with any pointwise stage between them
// exactly as the radix-2 pair does, in half the barriers.  N = I/2 complex
// points per array, `narr` arrays back to back; tw[k] = exp(-2 pi i k / I)
// for k < I/2 (shared or global memory), exp(-2 pi i k / I) = -tw[k - I/2]
// above.  DIF stage of span L (quarter Q = L/4), butterfly (a, b, c, d) at
// (i0, i0 + Q, i0 + 2Q, i0 + 3Q), s = -i (forward) or +i (inverse):
//   (a + c) + (b + d),  [(a - c) + s (b - d)] w^j,  [(a + c) - (b + d)] w^2j,  [(a - c) - s (b - d)] w^3j
// with w = exp(-/+ 2 pi i / L); the DIT stage applies the twiddles first.
template <class C> __device__ __forceinline__ C tw_at(const C* tw, int k, int half) {
    if (k < half) return tw[k];
    const C w = tw[k - half];
    return mkc(-w.x, -w.y);
}
template <class C> __device__ __forceinline__ C times_s(C z, bool inverse) {  // s z, s = +i or -i
    return inverse ? mkc(-z.y, z.x) : mkc(z.y, -z.x);
}
template <class C> __device__ __forceinline__ C maybe_conj(C w, bool inverse) { return inverse ? cconj(w) : w; }

template <class C>
__device__ void fft4_dif(C* x, int narr, int N, int logN, const C* tw, int I, bool inverse) {
    const int half = I >> 1;
    int L = N, logL = logN;
    if (logN & 1) {
        const int H = N >> 1;
        for (int t = threadIdx.x; t < narr * H; t += blockDim.x) {
            const int ar = t >> (logN - 1), j = t & (H - 1);
            C* xa = x + ar * N;
            const C w = maybe_conj(tw[2 * j], inverse);
            const C u = xa[j], v = xa[j + H];
            xa[j] = cadd(u, v);
            xa[j + H] = cmul(csub(u, v), w);
        }
        __syncthreads();
        L >>= 1;
        --logL;
    }
    for (; L >= 4; L >>= 2, logL -= 2) {
        const int Q = L >> 2, logQ = logL - 2;
        const int st = I >> logL;
        for (int t = threadIdx.x; t < narr * (N >> 2); t += blockDim.x) {
            const int ar = t >> (logN - 2), r = t & ((N >> 2) - 1);
            const int g = r >> logQ, j = r & (Q - 1);
            C* xa = x + ar * N + g * L + j;
            const C a = xa[0], b = xa[Q], c = xa[2 * Q], d = xa[3 * Q];
            const C apc = cadd(a, c), amc = csub(a, c), bpd = cadd(b, d), sbmd = times_s(csub(b, d), inverse);
            xa[0] = cadd(apc, bpd);
            xa[Q] = cmul(cadd(amc, sbmd), maybe_conj(tw_at(tw, j * st, half), inverse));
            xa[2 * Q] = cmul(csub(apc, bpd), maybe_conj(tw_at(tw, 2 * j * st, half), inverse));
            xa[3 * Q] = cmul(csub(amc, sbmd), maybe_conj(tw_at(tw, 3 * j * st, half), inverse));
        }
        __syncthreads();
    }
}

template <class C>
__device__ void fft4_dit(C* x, int narr, int N, int logN, const C* tw, int I, bool inverse) {
    const int half = I >> 1;
    const int top = (logN & 1) ? logN - 1 : logN;
    for (int logL = 2; logL <= top; logL += 2) {
        const int L = 1 << logL, Q = L >> 2, logQ = logL - 2;
        const int st = I >> logL;
        for (int t = threadIdx.x; t < narr * (N >> 2); t += blockDim.x) {
            const int ar = t >> (logN - 2), r = t & ((N >> 2) - 1);
            const int g = r >> logQ, j = r & (Q - 1);
            C* xa = x + ar * N + g * L + j;
            const C a = xa[0];
            const C b = cmul(xa[Q], maybe_conj(tw_at(tw, j * st, half), inverse));
            const C c = cmul(xa[2 * Q], maybe_conj(tw_at(tw, 2 * j * st, half), inverse));
            const C d = cmul(xa[3 * Q], maybe_conj(tw_at(tw, 3 * j * st, half), inverse));
            const C apc = cadd(a, c), amc = csub(a, c), bpd = cadd(b, d), sbmd = times_s(csub(b, d), inverse);
            xa[0] = cadd(apc, bpd);
            xa[Q] = cadd(amc, sbmd);
            xa[2 * Q] = csub(apc, bpd);
            xa[3 * Q] = csub(amc, sbmd);
        }
        __syncthreads();
    }
    if (logN & 1) {
        const int H = N >> 1;
        for (int t = threadIdx.x; t < narr * H; t += blockDim.x) {
            const int ar = t >> (logN - 1), j = t & (H - 1);
            C* xa = x + ar * N;
            const C w = maybe_conj(tw[2 * j], inverse);
            const C u = xa[j], v = cmul(xa[j + H], w);
            xa[j] = cadd(u, v);
            xa[j + H] = csub(u, v);
        }
        __syncthreads();
    }
}

// Real DFTs of length I through complex DFTs of length I/2 over the packed
// samples z_k = x_{2k} + i x_{2k+1} of ONE real row (packing two different
// fields would tie the smaller field's rounding error to the larger one).
// Stored coefficients F[0..R] (R < I/2) of a real row; Im F_0 is ignored.
template <class C> __device__ __forceinline__ C coef(const C* __restrict__ F, int m, int R) {
    if (m == 0) return mkc(F[0].x, decltype(F[0].x)(0));
    if (m <= R) return F[m];
    return mkc(decltype(F[0].x)(0), decltype(F[0].x)(0));
}

// Packed spectrum Z_k (k < I/2) whose unnormalised inverse DFT of length I/2
// is z_k = x_{2k} + i x_{2k+1}, x_n = sum_m X_m e^{2 pi i m n / I} (X Hermitian):
// Z_k = (X_k + conj X_{I/2-k}) + i (X_k - conj X_{I/2-k}) e^{+2 pi i k / I}.
template <class C>
__device__ __forceinline__ C irfft_pack(const C* __restrict__ F, int k, int R, int Hn, const C* __restrict__ tw) {
    const C a = coef(F, k, R);
    const C c = cconj(coef(F, Hn - k, R));
    const C s = cadd(a, c);
    const C d = cmul(csub(a, c), cconj(__ldg(&tw[k])));
    return mkc(s.x - d.y, s.y + d.x);
}

// X_m = E_m + e^{-2 pi i m / I} O_m from the forward DFT Z of the packed row,
// E_m = (Z_m + conj Z_{I/2-m}) / 2, O_m = (Z_m - conj Z_{I/2-m}) / (2 i).
template <class C> __device__ __forceinline__ C rfft_unpack(const C* z, int m, int Hn, const C* __restrict__ tw) {
    using T = decltype(z[0].x);
    const C Z = z[m];
    const C Zc = cconj(z[(Hn - m) & (Hn - 1)]);
    const C E = mkc(T(0.5) * (Z.x + Zc.x), T(0.5) * (Z.y + Zc.y));
    const C dz = csub(Z, Zc);
    const C O = mkc(T(0.5) * dz.y, T(-0.5) * dz.x);
    return cadd(E, cmul(__ldg(&tw[m]), O));
}

}  // namespace mlsdc
