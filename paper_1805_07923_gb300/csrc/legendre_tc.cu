// Tensor-core Legendre contractions for MLSDC_TF32 and MLSDC_BF16X3 on
// sm_103a: tcgen05.mma with accumulators in tensor memory, operands staged in
// shared memory by TMA (cp.async.bulk.tensor, 128-byte swizzle).
//
// Synthesis (Eq. spectral_to_physical_space, the Legendre sum per m), one CTA
// per zonal wavenumber m:
//   D[lat, c] = sum_k A[lat, k] B[c, k],  A = P^m_{m+k}(mu_lat) or H^m_{m+k},
//   M = 128 northern latitudes (zero padded), K = degrees n - m (padded),
//   N = 16 columns: the real and imaginary parts of the coefficients
//   (zeta, Phi', chi, psi for P; psi, chi for H) in two column groups, one
//   holding the even-(n-m) coefficients and one the odd ones, so that
//   north = even + odd and south = even - odd (H: odd - even).
// Analysis (Eq. legendre_transform), one CTA per (m, 128 degrees):
//   D[k, c] = sum_lat A[k, lat] B[c, lat],  A = P or H rows, K = latitudes,
//   B = the weighted Fourier coefficients of A..E combined north + south
//   (even) and north - south (odd); each row picks its parity's columns.
// TF32: operands rounded to tf32 (round to nearest); BF16X3: x = hi + lo in
// bf16 and D += A_hi B_hi + A_hi B_lo + A_lo B_hi.  Accumulation is float32
// in tensor memory; the final combination of F_E is float64.
//
// Every wait is bounded; on timeout the kernel records an error code in
// device memory (read by sh_plan_device_error), releases its tensor memory and
// returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <vector>

#include "complex.cuh"
#include "internal.h"
#include "rhs_kernels.cuh"  // coriolis_linear

namespace mlsdc {
namespace {

constexpr int kTcThreads = 128;
constexpr int kTileRows = 128;   // MMA M
constexpr int kTcN = 16;         // MMA N per column group
constexpr uint32_t kTmemCols = 32;
constexpr int kMaxKS = 192;      // synthesis K limit (R + 1 <= 192)
constexpr int kTileBytes = 16384;  // 128 rows x 128 B
constexpr uint32_t kSpinLimit = 1u << 24;
constexpr int kErrTmaTimeout = 1, kErrMmaTimeout = 2;

enum { MODE_TF32 = 0, MODE_BF16X3 = 1 };

struct Maps {
    CUtensorMap m[4];
};

struct TcState {
    int mode = 0;
    int KS = 0;   // padded synthesis K (multiple of 64)
    int J2p = 0;  // padded analysis K (multiple of 64)
    void* syn[4] = {nullptr, nullptr, nullptr, nullptr};
    void* ana[4] = {nullptr, nullptr, nullptr, nullptr};
    Maps map_syn, map_ana;
    int* d_err = nullptr;
    int2* d_tiles = nullptr;
    int n_tiles = 0;
    size_t smem_syn = 0, smem_ana = 0;
};

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t sa(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (uint32_t i = 0; i < kSpinLimit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kTmemCols) : "memory");
}

// K-major operand tile written by TMA with the 128-byte swizzle: rows of
// 128 B, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// K-major operand built by threads without swizzle: 8 x 16 B core matrices,
// `lbo` bytes apart along K and `sbo` bytes apart along N.
__device__ __forceinline__ uint64_t desc_plain(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           ((uint64_t)1 << 46);
}

// Instruction descriptors: D float32, A and B of one type (tf32, or bf16),
// both K-major, N = 16, M = 128.
constexpr uint32_t kIdescTf32 = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                                ((uint32_t)(kTileRows >> 4) << 24);
constexpr uint32_t kIdescBf16 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                                ((uint32_t)(kTileRows >> 4) << 24);

template <int MODE>
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
    if (MODE == MODE_TF32) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
            "l"(a), "l"(b), "r"(kIdescTf32), "r"(acc)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
            "l"(a), "l"(b), "r"(kIdescBf16), "r"(acc)
            : "memory");
    }
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
// 16 consecutive float32 columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// Store one B-operand value (row c of N = 16, column k) in the plain K-major
// layout: byte offset (k / kc) * 256 + (c / 8) * 128 + (c % 8) * 16 + (k % kc) * esz.
template <int MODE>
__device__ __forceinline__ void put_b(unsigned char* hi, unsigned char* lo, int c, int k, float v) {
    if (MODE == MODE_TF32) {
        const int off = (k >> 2) * 256 + (c >> 3) * 128 + (c & 7) * 16 + (k & 3) * 4;
        *reinterpret_cast<uint32_t*>(hi + off) = to_tf32(v);
    } else {
        const int off = (k >> 3) * 256 + (c >> 3) * 128 + (c & 7) * 16 + (k & 7) * 2;
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
        *reinterpret_cast<__nv_bfloat16*>(hi + off) = h;
        *reinterpret_cast<__nv_bfloat16*>(lo + off) = l;
    }
}

// ------------------------------------------------------------ shared layout
template <int MODE>
struct Shape {
    static constexpr int KB = MODE == MODE_TF32 ? 32 : 64;     // elements per 128-B K block
    static constexpr int KSTEP = MODE == MODE_TF32 ? 8 : 16;   // K per MMA
    static constexpr int ESZ = MODE == MODE_TF32 ? 4 : 2;
    static constexpr int NT = MODE == MODE_TF32 ? 2 : 4;       // A tables (P, H) or (P hi, P lo, H hi, H lo)
    static constexpr int NPART = MODE == MODE_TF32 ? 1 : 2;    // B parts (hi, lo)
    // bytes of one B operand (16 rows) for K elements
    static constexpr int b_bytes(int K) { return K * kTcN * ESZ; }
};

template <int MODE>
__host__ __device__ inline size_t tc_smem_bytes(int nkb_max) {
    using S = Shape<MODE>;
    return 1024 + (size_t)S::NT * nkb_max * kTileBytes + (size_t)2 * S::NPART * S::b_bytes(nkb_max * S::KB) + 64;
}

// ---------------------------------------------------------------- synthesis
template <int MODE>
__global__ void __launch_bounds__(kTcThreads, 1) k_tc_synth(const double2* __restrict__ state,
                                                            const __grid_constant__ Maps maps, int R, int J2, int nc,
                                                            double a, float2* __restrict__ four, int* __restrict__ err) {
    using S = Shape<MODE>;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int m = blockIdx.x;
    const int nm = R + 1 - m;
    const int off = m * (R + 1) - m * (m - 1) / 2;
    const int nkb = (nm + S::KB - 1) / S::KB;
    const int Kp = nkb * S::KB;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char* A = smem;                                   // [NT][nkb][16 KB]
    unsigned char* B = A + (size_t)S::NT * nkb * kTileBytes;  // [group][part][b_bytes(Kp)]
    const int bsz = S::b_bytes(Kp);
    uint64_t* bars = reinterpret_cast<uint64_t*>(B + 2 * S::NPART * bsz);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 2);
    volatile int* issued = reinterpret_cast<volatile int*>(tslot + 1);
    const uint32_t bar_tma = sa(&bars[0]), bar_mma = sa(&bars[1]);

    if (tid == 0) {
        mbar_init(bar_tma, 1);
        mbar_init(bar_mma, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(sa(tslot));
    __syncthreads();
    if (tid == 0) {
        mbar_expect_tx(bar_tma, (uint32_t)(S::NT * nkb * kTileBytes));
        for (int t = 0; t < S::NT; ++t)
            for (int kb = 0; kb < nkb; ++kb)
                tma_load_2d(sa(A + ((size_t)t * nkb + kb) * kTileBytes), &maps.m[t], kb * S::KB, m * kTileRows,
                            bar_tma);
    }
    // B operands: P group columns (zeta, Phi', chi, psi) x (re, im) + 8 x parity,
    //             H group columns (psi, chi) x (re, im) + 8 x parity (4..7, 12..15 zero)
    unsigned char* BP = B;
    unsigned char* BH = B + S::NPART * bsz;
    const double sa2 = -a * a;
    for (int k = tid; k < Kp; k += kTcThreads) {
        float pv[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        const int par = k & 1;
        if (k < nm) {
            const int n = m + k;
            const double s = n > 0 ? sa2 / (n * (n + 1.0)) : 0.0;
            const double2 ph = state[off + k], ze = state[nc + off + k], de = state[2 * nc + off + k];
            pv[0] = (float)ze.x; pv[1] = (float)ze.y;
            pv[2] = (float)ph.x; pv[3] = (float)ph.y;
            pv[4] = (float)(de.x * s); pv[5] = (float)(de.y * s);
            pv[6] = (float)(ze.x * s); pv[7] = (float)(ze.y * s);
        }
        for (int c = 0; c < 16; ++c) {
            const int comp = c & 7, cpar = c >> 3;
            const float vP = cpar == par ? pv[comp] : 0.f;
            const float vH = (cpar == par && comp < 4) ? pv[comp < 2 ? comp + 6 : comp + 2] : 0.f;
            put_b<MODE>(BP, BP + bsz, c, k, vP);
            put_b<MODE>(BH, BH + bsz, c, k, vH);
        }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    if (tid == 0) {
        *issued = 0;
        if (!mbar_wait(bar_tma, 0)) {
            atomicExch(err, kErrTmaTimeout);
        } else {
            *issued = 1;
            tc_fence_after();
            const int nsteps = Kp / S::KSTEP;
            for (int s = 0; s < nsteps; ++s) {
                const int kb = (s * S::KSTEP) / S::KB;
                const uint32_t ain = (uint32_t)((s * S::KSTEP) % S::KB) * S::ESZ;
                const uint32_t boff = (uint32_t)s * 512;
                for (int g = 0; g < 2; ++g) {
                    const uint32_t d = tmem + (uint32_t)(g * kTcN);
                    unsigned char* Bg = g == 0 ? BP : BH;
                    if (MODE == MODE_TF32) {
                        const uint64_t ad = desc_sw128(sa(A + ((size_t)g * nkb + kb) * kTileBytes) + ain);
                        const uint64_t bd = desc_plain(sa(Bg) + boff, 256, 128);
                        mma<MODE>(d, ad, bd, s > 0);
                    } else {
                        const uint64_t ah = desc_sw128(sa(A + ((size_t)(2 * g) * nkb + kb) * kTileBytes) + ain);
                        const uint64_t al = desc_sw128(sa(A + ((size_t)(2 * g + 1) * nkb + kb) * kTileBytes) + ain);
                        const uint64_t bh = desc_plain(sa(Bg) + boff, 256, 128);
                        const uint64_t bl = desc_plain(sa(Bg + bsz) + boff, 256, 128);
                        mma<MODE>(d, ah, bh, s > 0);
                        mma<MODE>(d, ah, bl, 1);
                        mma<MODE>(d, al, bh, 1);
                    }
                }
            }
            mma_commit(bar_mma);
        }
    }
    __syncthreads();
    const bool ok = *issued && mbar_wait(bar_mma, 0);
    if (*issued && !ok && lane == 0) atomicExch(err, kErrMmaTimeout);
    tc_fence_after();
    float vP[16], vH[16];
    const uint32_t lane_base = tmem + ((uint32_t)(32 * warp) << 16);
    tmem_ld16(lane_base, vP);
    tmem_ld16(lane_base + kTcN, vH);
    const int j = 32 * warp + lane;
    if (ok && j < J2) {
        const float ia = (float)(1.0 / a), dm = (float)m;
        const int J = 2 * J2, jS = J - 1 - j;
        const size_t fs = (size_t)J * (R + 1);
        auto cx = [&](const float* v, int c) { return make_float2(v[c], v[c + 1]); };
        // even parts at columns c, odd parts at c + 8
        const float2 zN = cadd(cx(vP, 0), cx(vP, 8)), zS = csub(cx(vP, 0), cx(vP, 8));
        const float2 pN = cadd(cx(vP, 2), cx(vP, 10)), pS = csub(cx(vP, 2), cx(vP, 10));
        const float2 xPN = cadd(cx(vP, 4), cx(vP, 12)), xPS = csub(cx(vP, 4), cx(vP, 12));
        const float2 sPN = cadd(cx(vP, 6), cx(vP, 14)), sPS = csub(cx(vP, 6), cx(vP, 14));
        const float2 sHN = cadd(cx(vH, 0), cx(vH, 8)), sHS = csub(cx(vH, 8), cx(vH, 0));
        const float2 xHN = cadd(cx(vH, 2), cx(vH, 10)), xHS = csub(cx(vH, 10), cx(vH, 2));
        four[0 * fs + (size_t)j * (R + 1) + m] = zN;
        four[0 * fs + (size_t)jS * (R + 1) + m] = zS;
        four[1 * fs + (size_t)j * (R + 1) + m] = pN;
        four[1 * fs + (size_t)jS * (R + 1) + m] = pS;
        four[2 * fs + (size_t)j * (R + 1) + m] = cscale(csub(cim(dm, xPN), sHN), ia);
        four[2 * fs + (size_t)jS * (R + 1) + m] = cscale(csub(cim(dm, xPS), sHS), ia);
        four[3 * fs + (size_t)j * (R + 1) + m] = cscale(cadd(cim(dm, sPN), xHN), ia);
        four[3 * fs + (size_t)jS * (R + 1) + m] = cscale(cadd(cim(dm, sPS), xHS), ia);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem);
}

// ----------------------------------------------------------------- analysis
template <int MODE>
__global__ void __launch_bounds__(kTcThreads, 1) k_tc_anal(const float2* __restrict__ four_out,
                                                           const __grid_constant__ Maps maps,
                                                           const int2* __restrict__ tiles, int R, int J2, int nc,
                                                           int J2p, double a, double2* __restrict__ FE,
                                                           const double2* __restrict__ state, double two_omega,
                                                           const double* __restrict__ cor,
                                                           int* __restrict__ err) {
    using S = Shape<MODE>;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int2 tl = tiles[blockIdx.x];
    const int m = tl.x, t = tl.y;
    const int nm = R + 1 - m;
    const int off = m * (R + 1) - m * (m - 1) / 2;
    const int nkb = (J2p + S::KB - 1) / S::KB;
    const int Kp = nkb * S::KB;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char* A = smem;
    unsigned char* B = A + (size_t)S::NT * nkb * kTileBytes;
    const int bsz = S::b_bytes(Kp);
    uint64_t* bars = reinterpret_cast<uint64_t*>(B + 2 * S::NPART * bsz);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 2);
    volatile int* issued = reinterpret_cast<volatile int*>(tslot + 1);
    const uint32_t bar_tma = sa(&bars[0]), bar_mma = sa(&bars[1]);

    if (tid == 0) {
        mbar_init(bar_tma, 1);
        mbar_init(bar_mma, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(sa(tslot));
    __syncthreads();
    if (tid == 0) {
        mbar_expect_tx(bar_tma, (uint32_t)(S::NT * nkb * kTileBytes));
        for (int q = 0; q < S::NT; ++q)
            for (int kb = 0; kb < nkb; ++kb)
                tma_load_2d(sa(A + ((size_t)q * nkb + kb) * kTileBytes), &maps.m[q], kb * S::KB,
                            off + t * kTileRows, bar_tma);
    }
    // B operands over latitudes: P group (C, A, B, E) x (re, im) + 8 x parity;
    // H group (D, B, A) x (re, im) + 8 x parity (columns 6, 7, 14, 15 zero).
    // even = north + south, odd = north - south.
    unsigned char* BP = B;
    unsigned char* BH = B + S::NPART * bsz;
    const int J = 2 * J2;
    const size_t fs = (size_t)J * (R + 1);
    for (int j = tid; j < Kp; j += kTcThreads) {
        float2 e[5], o[5];
        for (int f = 0; f < 5; ++f) {
            if (j < J2) {
                const float2 gN = four_out[(size_t)f * fs + (size_t)j * (R + 1) + m];
                const float2 gS = four_out[(size_t)f * fs + (size_t)(J - 1 - j) * (R + 1) + m];
                e[f] = cadd(gN, gS);
                o[f] = csub(gN, gS);
            } else {
                e[f] = o[f] = make_float2(0.f, 0.f);
            }
        }
        // field order in four_out: A, B, C, D, E
        const int pf[4] = {2, 0, 1, 4};   // C, A, B, E
        const int hf[3] = {3, 1, 0};      // D, B, A
        for (int c = 0; c < 16; ++c) {
            const int comp = c & 7, cpar = c >> 3;
            const float2* src = cpar ? o : e;
            const float2 zp = src[pf[comp >> 1]];
            const float vP = (comp & 1) ? zp.y : zp.x;
            float vH = 0.f;
            if (comp < 6) {
                const float2 zh = src[hf[comp >> 1]];
                vH = (comp & 1) ? zh.y : zh.x;
            }
            put_b<MODE>(BP, BP + bsz, c, j, vP);
            put_b<MODE>(BH, BH + bsz, c, j, vH);
        }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    if (tid == 0) {
        *issued = 0;
        if (!mbar_wait(bar_tma, 0)) {
            atomicExch(err, kErrTmaTimeout);
        } else {
            *issued = 1;
            tc_fence_after();
            const int nsteps = Kp / S::KSTEP;
            for (int s = 0; s < nsteps; ++s) {
                const int kb = (s * S::KSTEP) / S::KB;
                const uint32_t ain = (uint32_t)((s * S::KSTEP) % S::KB) * S::ESZ;
                const uint32_t boff = (uint32_t)s * 512;
                for (int g = 0; g < 2; ++g) {
                    const uint32_t d = tmem + (uint32_t)(g * kTcN);
                    unsigned char* Bg = g == 0 ? BP : BH;
                    if (MODE == MODE_TF32) {
                        const uint64_t ad = desc_sw128(sa(A + ((size_t)g * nkb + kb) * kTileBytes) + ain);
                        mma<MODE>(d, ad, desc_plain(sa(Bg) + boff, 256, 128), s > 0);
                    } else {
                        const uint64_t ah = desc_sw128(sa(A + ((size_t)(2 * g) * nkb + kb) * kTileBytes) + ain);
                        const uint64_t al = desc_sw128(sa(A + ((size_t)(2 * g + 1) * nkb + kb) * kTileBytes) + ain);
                        const uint64_t bh = desc_plain(sa(Bg) + boff, 256, 128);
                        const uint64_t bl = desc_plain(sa(Bg + bsz) + boff, 256, 128);
                        mma<MODE>(d, ah, bh, s > 0);
                        mma<MODE>(d, ah, bl, 1);
                        mma<MODE>(d, al, bh, 1);
                    }
                }
            }
            mma_commit(bar_mma);
        }
    }
    __syncthreads();
    const bool ok = *issued && mbar_wait(bar_mma, 0);
    if (*issued && !ok && lane == 0) atomicExch(err, kErrMmaTimeout);
    tc_fence_after();
    float vP[16], vH[16];
    const uint32_t lane_base = tmem + ((uint32_t)(32 * warp) << 16);
    tmem_ld16(lane_base, vP);
    tmem_ld16(lane_base + kTcN, vH);
    const int k = t * kTileRows + 32 * warp + lane;
    if (ok && k < nm) {
        const int par = k & 1;
        const float* P8 = vP + 8 * par;        // C, A, B, E at this row's parity
        const float* H8 = vH + 8 * (par ^ 1);  // D, B, A at the opposite parity
        const double2 sC{P8[0], P8[1]}, sA{P8[2], P8[3]}, sB{P8[4], P8[5]}, sE{P8[6], P8[7]};
        const double2 hD{H8[0], H8[1]}, hB{H8[2], H8[3]}, hA{H8[4], H8[5]};
        const int n = m + k;
        const double ia = 1.0 / a, dm = (double)m;
        const double2 divCD = cscale(csub(cim(dm, sC), hD), ia);
        const double2 divAB = cscale(csub(cim(dm, sA), hB), ia);
        const double2 curlAB = cscale(cadd(cim(dm, sB), hA), ia);
        const double lap = n * (n + 1.0) * ia * ia;
        double2 f0 = make_double2(-divCD.x, -divCD.y);
        double2 f1 = make_double2(-divAB.x, -divAB.y);
        double2 f2 = make_double2(curlAB.x + lap * sE.x, curlAB.y + lap * sE.y);
        double2 dz, dd;  // the Coriolis part, exactly in float64 (grid products carry no f)
        coriolis_linear(state, cor, nc, R, m, n, off, a, two_omega, dz, dd);
        f1 = cadd(f1, dz);
        f2 = cadd(f2, dd);
        if (m == 0) f0.y = f1.y = f2.y = 0.0;
        FE[off + k] = f0;
        FE[nc + off + k] = f1;
        FE[2 * nc + off + k] = f2;
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem);
}

// ---------------------------------------------------------- table builders
// Synthesis tables, K-major in n: row (m, lat) of length KS.
template <int MODE>
__global__ void k_build_syn(const double* __restrict__ T, int R, int J2, int KS, void* hi, void* lo) {
    const size_t total = (size_t)(R + 1) * kTileRows * KS;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(i % KS);
        const int row = (int)(i / KS);
        const int m = row / kTileRows, j = row % kTileRows;
        const int nm = R + 1 - m;
        float v = 0.f;
        if (j < J2 && k < nm) v = (float)T[(size_t)(m * (R + 1) - m * (m - 1) / 2 + k) * J2 + j];
        if (MODE == MODE_TF32) {
            reinterpret_cast<uint32_t*>(hi)[i] = to_tf32(v);
        } else {
            const __nv_bfloat16 h = __float2bfloat16_rn(v);
            reinterpret_cast<__nv_bfloat16*>(hi)[i] = h;
            reinterpret_cast<__nv_bfloat16*>(lo)[i] = __float2bfloat16_rn(v - __bfloat162float(h));
        }
    }
}
// Analysis tables, K-major in latitude: row (m, n) of length J2p.
template <int MODE>
__global__ void k_build_ana(const double* __restrict__ T, int nc, int J2, int J2p, void* hi, void* lo) {
    const size_t total = (size_t)nc * J2p;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(i % J2p);
        const size_t row = i / J2p;
        const float v = j < J2 ? (float)T[row * J2 + j] : 0.f;
        if (MODE == MODE_TF32) {
            reinterpret_cast<uint32_t*>(hi)[i] = to_tf32(v);
        } else {
            const __nv_bfloat16 h = __float2bfloat16_rn(v);
            reinterpret_cast<__nv_bfloat16*>(hi)[i] = h;
            reinterpret_cast<__nv_bfloat16*>(lo)[i] = __float2bfloat16_rn(v - __bfloat162float(h));
        }
    }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 2-D tensor map over a row-major [rows][cols] table, box 128 B x 128 rows, 128-B swizzle.
bool make_map(CUtensorMap* map, void* base, int mode, uint64_t cols, uint64_t rows) {
    auto enc = get_encode();
    if (!enc) return false;
    const int esz = mode == MODE_TF32 ? 4 : 2;
    cuuint64_t dims[2] = {cols, rows};
    cuuint64_t strides[1] = {cols * esz};
    cuuint32_t box[2] = {(cuuint32_t)(128 / esz), (cuuint32_t)kTileRows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, mode == MODE_TF32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                     base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

TcState* st_of(sh_plan_t p) { return reinterpret_cast<TcState*>(p->mp.tc); }

template <int MODE>
mlsdc_status build_tables(sh_plan_t p, TcState* s) {
    const int esz = MODE == MODE_TF32 ? 4 : 2;
    const size_t nsyn = (size_t)(p->R + 1) * kTileRows * s->KS;
    const size_t nana = (size_t)p->nc * s->J2p;
    const int nparts = MODE == MODE_TF32 ? 1 : 2;
    for (int t = 0; t < 2; ++t)
        for (int q = 0; q < nparts; ++q) {
            MLSDC_CUDA(cudaMalloc(&s->syn[t * nparts + q], nsyn * esz));
            MLSDC_CUDA(cudaMalloc(&s->ana[t * nparts + q], nana * esz));
            p->mp.tc_bytes += (int64_t)(nsyn + nana) * esz;
        }
    for (int t = 0; t < 2; ++t) {
        const double* src = t == 0 ? p->d_P : p->d_H;
        void* sh = s->syn[t * nparts];
        void* sl = nparts == 2 ? s->syn[t * nparts + 1] : nullptr;
        void* ah = s->ana[t * nparts];
        void* al = nparts == 2 ? s->ana[t * nparts + 1] : nullptr;
        k_build_syn<MODE><<<1024, 256>>>(src, p->R, p->J2, s->KS, sh, sl);
        k_build_ana<MODE><<<1024, 256>>>(src, p->nc, p->J2, s->J2p, ah, al);
        MLSDC_LAUNCHED("k_build_tables");
    }
    MLSDC_CUDA(cudaDeviceSynchronize());
    for (int q = 0; q < 2 * nparts; ++q) {
        if (!make_map(&s->map_syn.m[q], s->syn[q], MODE, s->KS, (uint64_t)(p->R + 1) * kTileRows) ||
            !make_map(&s->map_ana.m[q], s->ana[q], MODE, s->J2p, (uint64_t)p->nc)) {
            set_error_text("cuTensorMapEncodeTiled failed or is unavailable");
            return MLSDC_ERR_CUDA;
        }
    }
    const int nkb_syn = s->KS / Shape<MODE>::KB;
    const int nkb_ana = s->J2p / Shape<MODE>::KB;
    s->smem_syn = tc_smem_bytes<MODE>(nkb_syn);
    s->smem_ana = tc_smem_bytes<MODE>(nkb_ana);
    mlsdc_status rs = raise_smem_limit((const void*)k_tc_synth<MODE>, s->smem_syn);
    if (rs == MLSDC_OK) rs = raise_smem_limit((const void*)k_tc_anal<MODE>, s->smem_ana);
    if (rs != MLSDC_OK) return rs;
    return MLSDC_OK;
}

}  // namespace

mlsdc_status tc_init(sh_plan_t p) {
    if (p->J2 > kTileRows || p->R + 1 > kMaxKS) {
        set_error_text("tensor-core precisions need nlat/2 <= 128 and R <= 191");
        return MLSDC_ERR_INVALID;
    }
    TcState* s = new TcState();
    p->mp.tc = s;
    s->mode = p->precision == MLSDC_TF32 ? MODE_TF32 : MODE_BF16X3;
    s->KS = (p->R + 1 + 63) / 64 * 64;
    s->J2p = (p->J2 + 63) / 64 * 64;
    MLSDC_CUDA(cudaMalloc((void**)&s->d_err, sizeof(int)));
    MLSDC_CUDA(cudaMemset(s->d_err, 0, sizeof(int)));
    std::vector<int2> tiles;
    for (int m = 0; m <= p->R; ++m)
        for (int t = 0; t * kTileRows < p->R + 1 - m; ++t) tiles.push_back(make_int2(m, t));
    s->n_tiles = (int)tiles.size();
    MLSDC_CUDA(cudaMalloc((void**)&s->d_tiles, tiles.size() * sizeof(int2)));
    MLSDC_CUDA(cudaMemcpy(s->d_tiles, tiles.data(), tiles.size() * sizeof(int2), cudaMemcpyHostToDevice));
    return s->mode == MODE_TF32 ? build_tables<MODE_TF32>(p, s) : build_tables<MODE_BF16X3>(p, s);
}

void tc_free(sh_plan_t p) {
    TcState* s = st_of(p);
    if (!s) return;
    for (int q = 0; q < 4; ++q) {
        cudaFree(s->syn[q]);
        cudaFree(s->ana[q]);
    }
    cudaFree(s->d_err);
    cudaFree(s->d_tiles);
    delete s;
    p->mp.tc = nullptr;
}

mlsdc_status tc_synth(sh_plan_t p, const double* state, double a, cudaStream_t st) {
    TcState* s = st_of(p);
    if (s->mode == MODE_TF32)
        k_tc_synth<MODE_TF32><<<p->R + 1, kTcThreads, s->smem_syn, st>>>(
            (const double2*)state, s->map_syn, p->R, p->J2, p->nc, a, p->mp.four_in, s->d_err);
    else
        k_tc_synth<MODE_BF16X3><<<p->R + 1, kTcThreads, s->smem_syn, st>>>(
            (const double2*)state, s->map_syn, p->R, p->J2, p->nc, a, p->mp.four_in, s->d_err);
    MLSDC_LAUNCHED("k_tc_synth");
    return MLSDC_OK;
}

mlsdc_status tc_anal(sh_plan_t p, double a, double* FE, const double* state, double two_omega, cudaStream_t st) {
    TcState* s = st_of(p);
    if (s->mode == MODE_TF32)
        k_tc_anal<MODE_TF32><<<s->n_tiles, kTcThreads, s->smem_ana, st>>>(
            p->mp.four_out, s->map_ana, s->d_tiles, p->R, p->J2, p->nc, s->J2p, a, (double2*)FE,
            (const double2*)state, two_omega, p->d_cor, s->d_err);
    else
        k_tc_anal<MODE_BF16X3><<<s->n_tiles, kTcThreads, s->smem_ana, st>>>(
            p->mp.four_out, s->map_ana, s->d_tiles, p->R, p->J2, p->nc, s->J2p, a, (double2*)FE,
            (const double2*)state, two_omega, p->d_cor, s->d_err);
    MLSDC_LAUNCHED("k_tc_anal");
    return MLSDC_OK;
}

mlsdc_status tc_error(sh_plan_t p, int* code) {
    TcState* s = st_of(p);
    *code = 0;
    if (!s) return MLSDC_OK;
    MLSDC_CUDA(cudaMemcpy(code, s->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    return MLSDC_OK;
}

}  // namespace mlsdc
