// Complex helpers and shared-memory real FFTs, templated on the real type
// (double for the float64 path, float for the mixed-precision path).
#pragma once

#include <cuda_runtime.h>

#include "vblock.cuh"

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
// points per array, `narr` arrays back to back.  DIF stage of span L
// (quarter Q = L/4), butterfly (a, b, c, d) at (i0, i0 + Q, i0 + 2Q, i0 + 3Q),
// s = -i (forward) or +i (inverse):
//   (a + c) + (b + d),  [(a - c) + s (b - d)] w^j,  [(a + c) - (b + d)] w^2j,  [(a - c) - s (b - d)] w^3j
// with w = exp(-/+ 2 pi i / L); the DIT stage applies the twiddles first.
//
// Storage: element a of an array sits at swz(a), an XOR swizzle inside each
// aligned group of 16 that spreads every stage's access pattern (runs of
// 16 consecutive indices, or groups of 4 at strides 4 and 16) over distinct
// shared-memory banks; every access of these arrays goes through swz.
// Twiddles come from a per-stage table (fft4_stage_twiddles) laid out
// [radix-2 stage: w^2j, j < N/2][each radix-4 stage of span L, largest
// first: w^j, w^2j, w^3j for j < L/4], N - 1 entries, so a stage reads
// consecutive entries.
__device__ __forceinline__ int swz(int a) {
    const int s = (a >> 4) & 3;
    return a ^ (s | (s << 2));
}
template <class C> __device__ __forceinline__ C tw_at(const C* tw, int k, int half) {
    if (k < half) return tw[k];
    const C w = tw[k - half];
    return mkc(-w.x, -w.y);
}
template <class C> __device__ __forceinline__ C times_s(C z, bool inverse) {  // s z, s = +i or -i
    return inverse ? mkc(-z.y, z.x) : mkc(z.y, -z.x);
}
template <class C> __device__ __forceinline__ C maybe_conj(C w, bool inverse) { return inverse ? cconj(w) : w; }

// Fill the stage table (N - 1 entries) from tw[k] = exp(-2 pi i k / I),
// k < I/2 (any memory space); the caller synchronises before use.  These
// three work over the threads of the (virtual) block bk.
template <class C>
__device__ __forceinline__ void fft4_stage_twiddles(const Blk& bk, C* tab, const C* __restrict__ tw, int N, int logN, int I) {
    const int half = I >> 1;
    int off = 0;
    if (logN & 1) {
        const int H = N >> 1;
        for (int j = bk.t; j < H; j += bk.nt) tab[j] = tw[2 * j];
        off = H;
    }
    for (int logL = (logN & 1) ? logN - 1 : logN; logL >= 2; logL -= 2) {
        const int Q = 1 << (logL - 2), st = I >> logL;
        for (int e = bk.t; e < 3 * Q; e += bk.nt) {
            const int q = e / Q + 1, j = e - (q - 1) * Q;
            tab[off + e] = tw_at(tw, q * j * st, half);
        }
        off += 3 * Q;
    }
}

// The butterflies of one pass over `narr` arrays.  When the block's
// threads are a multiple of the butterflies per array (nq = N/4, or N/2 for
// the radix-2 pass) every thread keeps the same butterfly position in each
// array it visits (arrays ar0, ar0 + astep, ...), so its swizzled offsets and
// twiddles are formed once per pass; otherwise per item.  The same items in
// the same order either way.
template <class C>
__device__ __forceinline__ void dif4_bfly(C* xa, int s0, int s1, int s2, int s3, C w1, C w2, C w3, bool inverse) {
    const C a = xa[s0], b = xa[s1], c = xa[s2], d = xa[s3];
    const C apc = cadd(a, c), amc = csub(a, c), bpd = cadd(b, d), sbmd = times_s(csub(b, d), inverse);
    xa[s0] = cadd(apc, bpd);
    xa[s1] = cmul(cadd(amc, sbmd), w1);
    xa[s2] = cmul(csub(apc, bpd), w2);
    xa[s3] = cmul(csub(amc, sbmd), w3);
}
template <class C>
__device__ __forceinline__ void dit4_bfly(C* xa, int s0, int s1, int s2, int s3, C w1, C w2, C w3, bool inverse) {
    const C a = xa[s0];
    const C b = cmul(xa[s1], w1);
    const C c = cmul(xa[s2], w2);
    const C d = cmul(xa[s3], w3);
    const C apc = cadd(a, c), amc = csub(a, c), bpd = cadd(b, d), sbmd = times_s(csub(b, d), inverse);
    xa[s0] = cadd(apc, bpd);
    xa[s1] = cadd(amc, sbmd);
    xa[s2] = csub(apc, bpd);
    xa[s3] = csub(amc, sbmd);
}
// one radix-4 pass of span L = 4 Q (twiddles tq: w^j, w^2j, w^3j blocks of Q)
template <class C, bool DIT>
__device__ __forceinline__ void pass4(const Blk& bk, C* x, int narr, int N, int logN, int L, int logQ, const C* tq,
                                      bool inverse) {
    const int Q = L >> 2, nq = N >> 2;
    if (bk.nt % nq == 0) {
        const int ar0 = bk.t >> (logN - 2);
        if (ar0 >= narr) return;  // no butterfly for this thread in this pass
        const int r = bk.t & (nq - 1), g = r >> logQ, j = r & (Q - 1), i0 = g * L + j;
        const int s0 = swz(i0), s1 = swz(i0 + Q), s2 = swz(i0 + 2 * Q), s3 = swz(i0 + 3 * Q);
        const C w1 = maybe_conj(tq[j], inverse), w2 = maybe_conj(tq[Q + j], inverse),
                w3 = maybe_conj(tq[2 * Q + j], inverse);
        const int astep = bk.nt >> (logN - 2);
        for (int ar = ar0; ar < narr; ar += astep) {
            if (DIT)
                dit4_bfly(x + ar * N, s0, s1, s2, s3, w1, w2, w3, inverse);
            else
                dif4_bfly(x + ar * N, s0, s1, s2, s3, w1, w2, w3, inverse);
        }
        return;
    }
    for (int t = bk.t; t < narr * nq; t += bk.nt) {
        const int ar = t >> (logN - 2), r = t & (nq - 1);
        const int g = r >> logQ, j = r & (Q - 1);
        const int i0 = g * L + j;
        const C w1 = maybe_conj(tq[j], inverse), w2 = maybe_conj(tq[Q + j], inverse),
                w3 = maybe_conj(tq[2 * Q + j], inverse);
        if (DIT)
            dit4_bfly(x + ar * N, swz(i0), swz(i0 + Q), swz(i0 + 2 * Q), swz(i0 + 3 * Q), w1, w2, w3, inverse);
        else
            dif4_bfly(x + ar * N, swz(i0), swz(i0 + Q), swz(i0 + 2 * Q), swz(i0 + 3 * Q), w1, w2, w3, inverse);
    }
}
// the radix-2 pass (odd log2 N): span N, twiddles tab[j], j < N/2
template <class C, bool DIT>
__device__ __forceinline__ void pass2(const Blk& bk, C* x, int narr, int N, int logN, const C* tab, bool inverse) {
    const int H = N >> 1;
    auto bfly = [&](C* xa, int j, int s0, int s1) {
        const C w = maybe_conj(tab[j], inverse);
        if (DIT) {
            const C u = xa[s0], v = cmul(xa[s1], w);
            xa[s0] = cadd(u, v);
            xa[s1] = csub(u, v);
        } else {
            const C u = xa[s0], v = xa[s1];
            xa[s0] = cadd(u, v);
            xa[s1] = cmul(csub(u, v), w);
        }
    };
    if (bk.nt % H == 0) {
        const int ar0 = bk.t >> (logN - 1);
        if (ar0 >= narr) return;
        const int j = bk.t & (H - 1), s0 = swz(j), s1 = swz(j + H), astep = bk.nt >> (logN - 1);
        for (int ar = ar0; ar < narr; ar += astep) bfly(x + ar * N, j, s0, s1);
        return;
    }
    for (int t = bk.t; t < narr * H; t += bk.nt) {
        const int ar = t >> (logN - 1), j = t & (H - 1);
        bfly(x + ar * N, j, swz(j), swz(j + H));
    }
}

template <class C>
__device__ __forceinline__ void fft4_dif(const Blk& bk, C* x, int narr, int N, int logN, const C* tab, bool inverse) {
    int L = N, logL = logN, off = 0;
    if (logN & 1) {
        pass2<C, false>(bk, x, narr, N, logN, tab, inverse);
        bk.sync();
        off = N >> 1;
        L >>= 1;
        --logL;
    }
    for (; L >= 4; L >>= 2, logL -= 2) {
        pass4<C, false>(bk, x, narr, N, logN, L, logL - 2, tab + off, inverse);
        bk.sync();
        off += 3 * (L >> 2);
    }
}

template <class C>
__device__ __forceinline__ void fft4_dit(const Blk& bk, C* x, int narr, int N, int logN, const C* tab, bool inverse) {
    const int top = (logN & 1) ? logN - 1 : logN;
    const int r2 = (logN & 1) ? (N >> 1) : 0;  // entries of the radix-2 stage
    for (int logL = 2; logL <= top; logL += 2) {
        // the table holds the radix-4 stages largest first: skip the larger spans
        int off = r2;
        for (int l2 = top; l2 > logL; l2 -= 2) off += 3 * (1 << (l2 - 2));
        pass4<C, true>(bk, x, narr, N, logN, 1 << logL, logL - 2, tab + off, inverse);
        bk.sync();
    }
    if (logN & 1) {
        pass2<C, true>(bk, x, narr, N, logN, tab, inverse);
        bk.sync();
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

// rfft_unpack for an array stored through swz (the fft4 storage).
template <class C> __device__ __forceinline__ C rfft_unpack_sw(const C* z, int m, int Hn, const C* __restrict__ tw) {
    using T = decltype(z[0].x);
    const C Z = z[swz(m)];
    const C Zc = cconj(z[swz((Hn - m) & (Hn - 1))]);
    const C E = mkc(T(0.5) * (Z.x + Zc.x), T(0.5) * (Z.y + Zc.y));
    const C dz = csub(Z, Zc);
    const C O = mkc(T(0.5) * dz.y, T(-0.5) * dz.x);
    return cadd(E, cmul(__ldg(&tw[m]), O));
}

}  // namespace mlsdc
