// Device side of the tensor-core Legendre contractions (legendre_tc.cu has
// the description, the tables and the launches): PTX helpers, the shared
// memory layout, the K loop, and the synthesis, analysis and
// warp-specialised analysis as bodies on a Blk (vblock.cuh) with their
// kernels.  The persistent ensemble kernel (persistent.cu) runs the same
// bodies.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "async_copy.cuh"
#include "complex.cuh"
#include "convert.cuh"
#include "internal.h"
#include "rhs_kernels.cuh"  // coriolis_linear, FourStride

namespace mlsdc {
namespace tc {

constexpr int kTcThreads = 128;
constexpr int kTileRows = 128;   // MMA M
constexpr int kMaxKS = 192;      // synthesis K limit (R + 1 <= 192)
constexpr int kTileBytes = 16384;  // 128 rows x 128 B


enum { MODE_TF32 = 0, MODE_BF16X3 = 1 };

struct Maps {
    CUtensorMap m[4];
};

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

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

// tcgen05.mma of one K step; the instruction descriptor carries D float32,
// A and B of one type (tf32, or bf16), both K-major, N and M = 128.
template <int MODE>
__device__ __forceinline__ void mma_n(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    if (MODE == MODE_TF32) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc)
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


// Store one B-operand value (row r of N rows, column k of one K block) in the
// plain K-major layout: byte offset (k / kc) * lbo + (r / 8) * 128 + (r % 8) * 16
// + (k % kc) * esz, kc = 16 / esz elements per core-matrix row, lbo = 16 N + 16
// (lbo_for): the extra 16 bytes shift consecutive K groups by four banks, so a
// warp writing one column for 32 consecutive k hits distinct banks.
template <int MODE>
__device__ __forceinline__ void put_b(unsigned char* hi, unsigned char* lo, int r, int k, float v, uint32_t lbo) {
    if (MODE == MODE_TF32) {
        const uint32_t off = (uint32_t)(k >> 2) * lbo + (r >> 3) * 128 + (r & 7) * 16 + (k & 3) * 4;
        *reinterpret_cast<uint32_t*>(hi + off) = to_tf32(v);
    } else {
        const uint32_t off = (uint32_t)(k >> 3) * lbo + (r >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
        *reinterpret_cast<__nv_bfloat16*>(hi + off) = h;
        *reinterpret_cast<__nv_bfloat16*>(lo + off) = l;
    }
}

// put_b for the KV = 16 / esz consecutive K values k = KV g ... KV g + KV - 1
// of row r, stored as one 16-byte word per part (same layout and rounding).
// Eight lanes storing one row for consecutive groups g hit distinct banks
// (the 16-byte shift of lbo_for).
template <int MODE>
__device__ __forceinline__ void put_bv(unsigned char* hi, unsigned char* lo, int r, int g, const float* v,
                                       uint32_t lbo) {
    const uint32_t off = (uint32_t)g * lbo + (r >> 3) * 128 + (r & 7) * 16;
    if (MODE == MODE_TF32) {
        *reinterpret_cast<uint4*>(hi + off) = make_uint4(to_tf32(v[0]), to_tf32(v[1]), to_tf32(v[2]), to_tf32(v[3]));
    } else {
        uint32_t h[4], l[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const __nv_bfloat162 hv = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
            const float2 hf = __bfloat1622float2(hv);
            const __nv_bfloat162 lv = __floats2bfloat162_rn(v[2 * q] - hf.x, v[2 * q + 1] - hf.y);
            h[q] = *reinterpret_cast<const uint32_t*>(&hv);
            l[q] = *reinterpret_cast<const uint32_t*>(&lv);
        }
        *reinterpret_cast<uint4*>(hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<uint4*>(lo + off) = make_uint4(l[0], l[1], l[2], l[3]);
    }
}

// ------------------------------------------------------------ shared layout
template <int MODE>
struct Shape {
    static constexpr int KB = MODE == MODE_TF32 ? 32 : 64;     // elements per 128-B K block
    static constexpr int KSTEP = MODE == MODE_TF32 ? 8 : 16;   // K per MMA
    static constexpr int NT = MODE == MODE_TF32 ? 2 : 4;       // A tables (P, H) or (P hi, P lo, H hi, H lo)
    static constexpr int NPART = MODE == MODE_TF32 ? 1 : 2;    // B parts (hi, lo)
    static constexpr int KV = MODE == MODE_TF32 ? 4 : 8;       // K values per 16-byte B word
};

// One pipeline stage: the A tiles of one K block, then the B tiles of the
// two column groups (P, H) for `chunk` members (16 rows each) and each part.
__host__ __device__ inline uint32_t lbo_for(int N) { return 16u * (uint32_t)N + 16u; }
// one B tile (8 core-matrix columns along K) for up to `chunk` members
__host__ __device__ inline size_t btile_bytes(int chunk) { return (size_t)8 * lbo_for(16 * chunk); }
__host__ __device__ inline size_t stage_bytes(int mode, int chunk) {
    const int nt = mode == MODE_TF32 ? 2 : 4, npart = mode == MODE_TF32 ? 1 : 2;
    const size_t b = (size_t)nt * kTileBytes + (size_t)2 * npart * btile_bytes(chunk);
    return (b + 1023) & ~(size_t)1023;  // the next stage's A tiles need 1024-byte alignment (128-byte swizzle)
}
__host__ __device__ inline size_t cta_smem_bytes(int mode, int chunk, int stages) {
    return 1024 + (size_t)stages * stage_bytes(mode, chunk) + 128;
}
__host__ __device__ inline uint32_t tmem_cols_for(int ncols) {
    uint32_t c = 32;
    while (c < (uint32_t)ncols) c <<= 1;
    return c;
}

struct TcArgs {
    int R, J2, nc, J2p, members, chunk, stages;
    double two_omega;
    const double2* state;
    size_t state_ms;      // member stride of the state (complex values)
    float2* four_in;      // synthesis output, member stride 4 J (R+1)
    const float2* four_out;  // analysis input, member stride 5 J (R+1)
    FourStride fo;           // layout of each four_out field
    double2* FE;
    size_t fe_ms;
    const double* cor;
    const int2* tiles;
    int n_tiles;
    int* err;
    // host-computed constants (no float64 division in the kernels)
    float ia_f, na2_f;       // 1/a, -a^2
    const float* invnn;      // [R+1] 1/(n(n+1)), 0 for n = 0
};

// Stage buffers, barriers and tensor memory of one CTA.
struct Cta {
    unsigned char* smem;
    size_t stage_sz;
    uint64_t* bars;  // [0, kMaxStages): TMA full; [kMaxStages, 2 kMaxStages): MMA done
    uint32_t* tslot;
    volatile int* abort;
};
constexpr int kMaxStages = 2;

template <int MODE>
__device__ inline Cta cta_setup(const Blk& bk, int chunk, int stages, uint32_t ncols) {
    Cta c;
    c.smem = (unsigned char*)(((uintptr_t)bk.smem + 1023) & ~(uintptr_t)1023);
    c.stage_sz = stage_bytes(MODE, chunk);
    c.bars = reinterpret_cast<uint64_t*>(c.smem + stages * c.stage_sz);
    c.tslot = reinterpret_cast<uint32_t*>(c.bars + 2 * kMaxStages);
    c.abort = reinterpret_cast<volatile int*>(c.tslot + 1);
    if (bk.t == 0) {
        for (int s = 0; s < 2 * kMaxStages; ++s) mbar_init(sa(&c.bars[s]), 1);
        *c.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if ((bk.t >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sa(c.tslot)),
                     "r"(ncols)
                     : "memory");
        // a CTA of the persistent kernel allocates again for later blocks
        if (!bk.persist) asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    bk.sync();
    tc_fence_after();
    return c;
}

template <int MODE>
__device__ __forceinline__ unsigned char* a_tile(const Cta& c, int st, int t) {
    return c.smem + st * c.stage_sz + (size_t)t * kTileBytes;
}
template <int MODE>
__device__ __forceinline__ unsigned char* b_tile(const Cta& c, int st, int grp, int part, int chunk) {
    using S = Shape<MODE>;
    return c.smem + st * c.stage_sz + (size_t)S::NT * kTileBytes + (size_t)(grp * S::NPART + part) * btile_bytes(chunk);
}

// Issue the four MMA steps of one K block for both column groups.
template <int MODE>
__device__ __forceinline__ void mma_block(const Cta& c, int st, int chunk, uint32_t tmem, int N, uint32_t idesc,
                                          bool first) {
    using S = Shape<MODE>;
    const uint32_t lbo = lbo_for(N);
    for (int s = 0; s < S::KB / S::KSTEP; ++s) {
        const uint32_t acc = (!first || s > 0) ? 1u : 0u;
        for (int grp = 0; grp < 2; ++grp) {
            const uint32_t d = tmem + (uint32_t)(grp * N);
            const uint32_t bofs = (uint32_t)s * 2 * lbo;
            if (MODE == MODE_TF32) {
                const uint64_t ad = desc_sw128(sa(a_tile<MODE>(c, st, grp)) + s * 32);
                const uint64_t bd = desc_plain(sa(b_tile<MODE>(c, st, grp, 0, chunk)) + bofs, lbo, 128);
                mma_n<MODE>(d, ad, bd, idesc, acc);
            } else {
                const uint64_t ah = desc_sw128(sa(a_tile<MODE>(c, st, 2 * grp)) + s * 32);
                const uint64_t al = desc_sw128(sa(a_tile<MODE>(c, st, 2 * grp + 1)) + s * 32);
                const uint64_t bh = desc_plain(sa(b_tile<MODE>(c, st, grp, 0, chunk)) + bofs, lbo, 128);
                const uint64_t bl = desc_plain(sa(b_tile<MODE>(c, st, grp, 1, chunk)) + bofs, lbo, 128);
                mma_n<MODE>(d, ah, bh, idesc, acc);
                mma_n<MODE>(d, ah, bl, idesc, 1u);
                mma_n<MODE>(d, al, bh, idesc, 1u);
            }
        }
    }
}

// The K loop shared by synthesis and analysis.  Stage st holds K block kb
// (st = kb % stages).  Before the threads overwrite a stage's B tiles and
// thread 0 reloads its A tiles, the MMAs that read it (K block kb - stages)
// must have completed; thread 0 issues the MMAs of a block once its TMA
// bytes have landed and the B tiles are written, then commits to the stage's
// MMA barrier.  build_b(st, kb) writes the B tiles of block kb; load_a(st,
// kb) issues its TMA loads.  Returns false if a wait gave up.
template <int MODE, class BuildB, class LoadA>
__device__ inline bool k_loop(const Blk& bk, const Cta& c, int nkb, int stages, int chunk, uint32_t tmem, int N, uint32_t idesc,
                              int* err, BuildB build_b, LoadA load_a) {
    if (bk.t == 0)
        for (int kb = 0; kb < nkb && kb < stages; ++kb) load_a(kb % stages, kb);
    // the table tiles are constant: their loads overlap the previous kernel;
    // the B operand depends on it
    pdl_wait();
    pdl_launch();
    for (int kb = 0; kb < nkb; ++kb) {
        const int st = kb % stages;
        const uint32_t use = (uint32_t)(kb / stages);
        if (kb >= stages) {
            if (!mbar_wait(sa(&c.bars[kMaxStages + st]), (use - 1) & 1)) {
                if ((bk.t & 31) == 0) atomicExch(err, kErrMmaTimeout);
                *c.abort = 1;
            }
            if (bk.t == 0 && !*c.abort) load_a(st, kb);
        }
        build_b(st, kb);
        fence_async_smem();
        tc_fence_before();
        bk.sync();
        tc_fence_after();
        if (*c.abort) return false;
        if (bk.t == 0) {
            if (!mbar_wait(sa(&c.bars[st]), use & 1)) {
                atomicExch(err, kErrTmaTimeout);
                *c.abort = 1;
            } else {
                tc_fence_after();
                mma_block<MODE>(c, st, chunk, tmem, N, idesc, kb == 0);
                mma_commit(sa(&c.bars[kMaxStages + st]));
            }
        }
        bk.sync();
        if (*c.abort) return false;
    }
    const int last = nkb - 1;
    if (!mbar_wait(sa(&c.bars[kMaxStages + last % stages]), (uint32_t)(last / stages) & 1)) {
        if ((bk.t & 31) == 0) atomicExch(err, kErrMmaTimeout);
        return false;
    }
    tc_fence_after();
    return true;
}

template <int MODE>
__device__ __forceinline__ uint32_t idesc_for(int N) {
    const uint32_t base = MODE == MODE_TF32 ? ((1u << 4) | (2u << 7) | (2u << 10)) : ((1u << 4) | (1u << 7) | (1u << 10));
    return base | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kTileRows >> 4) << 24);
}

// Free the block's tensor memory.  In the persistent kernel the block's
// shared memory then serves other bodies: its mbarriers (the four pipeline
// barriers, and with ws_bars the warp-specialised kernel's four accumulator
// barriers after them) are invalidated first.
__device__ __forceinline__ void cta_release(const Blk& bk, const Cta& c, uint32_t tmem, uint32_t ncols,
                                            bool ws_bars = false) {
    tc_fence_before();
    bk.sync();
    if ((bk.t >> 5) == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
    if (bk.persist && bk.t == 0) {
        for (int s = 0; s < 2 * kMaxStages; ++s) mbar_inval(sa(&c.bars[s]));
        if (ws_bars)
            for (int s = 8; s < 12; ++s) mbar_inval(sa(&c.bars[s]));
    }
}

// ---------------------------------------------------------------- synthesis
// grid (R + 1, member chunks): one zonal wavenumber m and up to `chunk`
// members per CTA; D[lat, 16 b + c] accumulates over the degrees of m.
template <int MODE>
__device__ __forceinline__ void b_tc_synth(const Blk& bk, const Maps& maps, const TcArgs& g) {
    using S = Shape<MODE>;
    const int m = bk.idx.x;
    const int b0 = bk.idx.y * g.chunk;
    const int bc = min(g.chunk, g.members - b0);
    const int N = 16 * bc;
    const int R = g.R, nm = R + 1 - m;
    const int off = m * (R + 1) - m * (m - 1) / 2;
    const int nkb = (nm + S::KB - 1) / S::KB;
    const uint32_t ncols = tmem_cols_for(2 * N);
    const Cta c = cta_setup<MODE>(bk, g.chunk, g.stages, ncols);
    const uint32_t tmem = *c.tslot;
    const uint32_t lbo = lbo_for(N);
    auto load_a = [&](int st, int kb) {
        mbar_expect_tx(sa(&c.bars[st]), (uint32_t)(S::NT * kTileBytes));
        for (int t = 0; t < S::NT; ++t)
            tma_load_2d(sa(a_tile<MODE>(c, st, t)), &maps.m[t], kb * S::KB, m * kTileRows, sa(&c.bars[st]));
    };
    // B columns per member b: P group (zeta, Phi', chi, psi) x (re, im) + 8 x parity,
    // H group (psi, chi) x (re, im) + 8 x parity (4..7 and 12..15 zero).
    // One work item per (member, group of KV degrees, quantity q = zeta,
    // Phi', chi, psi): KV consecutive coefficients, each target column
    // stored as one 16-byte word per part (K groups start at multiples of KV,
    // so the even columns take the even v and the odd columns the odd v).
    constexpr int KV = S::KV, NG = S::KB / S::KV;
    if (bk.t < 2 * bc) {  // the always-zero H columns, written once per stage buffer
        const float z[KV] = {};
        const int b = bk.t >> 1, col = (bk.t & 1) ? 12 : 4;
        for (int st = 0; st < g.stages; ++st)
            for (int gg = 0; gg < NG; ++gg)
                for (int cc = 0; cc < 4; ++cc)
                    put_bv<MODE>(b_tile<MODE>(c, st, 1, 0, g.chunk), b_tile<MODE>(c, st, 1, S::NPART - 1, g.chunk),
                                 16 * b + col + cc, gg, z, lbo);
    }
    auto build_b = [&](int st, int kb) {
        unsigned char* P0 = b_tile<MODE>(c, st, 0, 0, g.chunk);
        unsigned char* P1 = b_tile<MODE>(c, st, 0, S::NPART - 1, g.chunk);
        unsigned char* H0 = b_tile<MODE>(c, st, 1, 0, g.chunk);
        unsigned char* H1 = b_tile<MODE>(c, st, 1, S::NPART - 1, g.chunk);
        for (int it = bk.t; it < bc * 4 * NG; it += kTcThreads) {
            const int gg = it % NG, qb = it / NG;
            const int q = qb & 3, b = qb >> 2;
            const int k0 = kb * S::KB + gg * KV;
            // state fields: Phi' at 0, zeta at nc, delta at 2 nc
            const double2* x =
                g.state + (size_t)(b0 + b) * g.state_ms + (q == 1 ? 0 : q == 2 ? 2 * g.nc : g.nc) + off;
            float er[KV], ei[KV], orr[KV], oi[KV];
#pragma unroll
            for (int v = 0; v < KV; ++v) {
                const int kk = k0 + v;
                float xr = 0.f, xi = 0.f;
                if (kk < nm) {
                    const double2 z = x[kk];
                    xr = (float)z.x;
                    xi = (float)z.y;
                    if (q >= 2) {  // psi, chi = -a^2/(n(n+1)) (zeta, delta)
                        const float sc = g.na2_f * g.invnn[m + kk];
                        xr *= sc;
                        xi *= sc;
                    }
                }
                const bool odd = v & 1;
                er[v] = odd ? 0.f : xr;
                ei[v] = odd ? 0.f : xi;
                orr[v] = odd ? xr : 0.f;
                oi[v] = odd ? xi : 0.f;
            }
            const int r = 16 * b + 2 * q;
            put_bv<MODE>(P0, P1, r, gg, er, lbo);
            put_bv<MODE>(P0, P1, r + 1, gg, ei, lbo);
            put_bv<MODE>(P0, P1, r + 8, gg, orr, lbo);
            put_bv<MODE>(P0, P1, r + 9, gg, oi, lbo);
            if (q >= 2) {  // H columns: psi at 0, 1; chi at 2, 3
                const int rh = 16 * b + (q == 3 ? 0 : 2);
                put_bv<MODE>(H0, H1, rh, gg, er, lbo);
                put_bv<MODE>(H0, H1, rh + 1, gg, ei, lbo);
                put_bv<MODE>(H0, H1, rh + 8, gg, orr, lbo);
                put_bv<MODE>(H0, H1, rh + 9, gg, oi, lbo);
            }
        }
    };
    const bool ok = k_loop<MODE>(bk, c, nkb, g.stages, g.chunk, tmem, N, idesc_for<MODE>(N), g.err, build_b, load_a);
    const int warp = bk.t >> 5, lane = bk.t & 31;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * warp) << 16);
    const int j = 32 * warp + lane;
    const int J = 2 * g.J2, jS = J - 1 - j;
    const size_t fs = (size_t)J * (R + 1);
    const size_t iN = (size_t)j * (R + 1) + m, iS = (size_t)jS * (R + 1) + m;
    for (int b = 0; b < bc; ++b) {
        float vP[16], vH[16];
        tmem_ld16(lane_base + 16 * b, vP);
        tmem_ld16(lane_base + N + 16 * b, vH);
        if (!ok || j >= g.J2) continue;
        float2* four = g.four_in + (size_t)(b0 + b) * 4 * fs;
        const float ia = g.ia_f, dm = (float)m;
        auto cx = [&](const float* v, int q) { return make_float2(v[q], v[q + 1]); };
        // even parts at columns q, odd parts at q + 8
        const float2 zN = cadd(cx(vP, 0), cx(vP, 8)), zS = csub(cx(vP, 0), cx(vP, 8));
        const float2 pN = cadd(cx(vP, 2), cx(vP, 10)), pS = csub(cx(vP, 2), cx(vP, 10));
        const float2 xPN = cadd(cx(vP, 4), cx(vP, 12)), xPS = csub(cx(vP, 4), cx(vP, 12));
        const float2 sPN = cadd(cx(vP, 6), cx(vP, 14)), sPS = csub(cx(vP, 6), cx(vP, 14));
        const float2 sHN = cadd(cx(vH, 0), cx(vH, 8)), sHS = csub(cx(vH, 8), cx(vH, 0));
        const float2 xHN = cadd(cx(vH, 2), cx(vH, 10)), xHS = csub(cx(vH, 10), cx(vH, 2));
        four[0 * fs + iN] = zN;
        four[0 * fs + iS] = zS;
        four[1 * fs + iN] = pN;
        four[1 * fs + iS] = pS;
        four[2 * fs + iN] = cscale(csub(cim(dm, xPN), sHN), ia);
        four[2 * fs + iS] = cscale(csub(cim(dm, xPS), sHS), ia);
        four[3 * fs + iN] = cscale(cadd(cim(dm, sPN), xHN), ia);
        four[3 * fs + iS] = cscale(cadd(cim(dm, sPS), xHS), ia);
    }
    cta_release(bk, c, tmem, ncols);
}

// ----------------------------------------------------------------- analysis
// grid (tiles, member chunks): one (m, 128 degrees) tile and up to `chunk`
// members per CTA; D[k, 16 b + c] accumulates over the latitudes.
template <int MODE>
__device__ __forceinline__ void b_tc_anal(const Blk& bk, const Maps& maps, const TcArgs& g) {
    using S = Shape<MODE>;
    const int2 tl = g.tiles[bk.idx.x];
    const int m = tl.x, t = tl.y;
    const int b0 = bk.idx.y * g.chunk;
    const int bc = min(g.chunk, g.members - b0);
    const int N = 16 * bc;
    const int R = g.R, nm = R + 1 - m;
    const int off = m * (R + 1) - m * (m - 1) / 2;
    const int nkb = (g.J2p + S::KB - 1) / S::KB;
    const uint32_t ncols = tmem_cols_for(2 * N);
    const Cta c = cta_setup<MODE>(bk, g.chunk, g.stages, ncols);
    const uint32_t tmem = *c.tslot;
    const uint32_t lbo = lbo_for(N);
    const int J = 2 * g.J2;
    const size_t fs = (size_t)J * (R + 1);
    auto load_a = [&](int st, int kb) {
        mbar_expect_tx(sa(&c.bars[st]), (uint32_t)(S::NT * kTileBytes));
        for (int q = 0; q < S::NT; ++q)
            tma_load_2d(sa(a_tile<MODE>(c, st, q)), &maps.m[q], kb * S::KB, off + t * kTileRows, sa(&c.bars[st]));
    };
    // B columns per member over latitudes: P group (C, A, B, E) x (re, im) + 8 x parity,
    // H group (D, B, A) x (re, im) + 8 x parity (6, 7, 14, 15 zero);
    // even = north + south, odd = north - south.
    // m-contiguous input (launches of one or two members): one item per
    // (member, latitude), one value per store, 64 threads busy per member.
    // Latitude-contiguous input (more members): one item per (member, group
    // of KV latitudes, field), two runs of KV latitudes (north and the
    // mirrored south) read as 16-byte words, each target column stored as
    // one 16-byte word per part; the eight lanes of a quarter warp take
    // consecutive latitude groups, which the K-group stride (16 N + 16 bytes)
    // puts in distinct banks.  With few members the longer per-item work of
    // the second form measured slower; with many its fewer loads and stores win.
    const FourStride fx = g.fo;
    const bool lat_contig = fx.sj == 1;
    constexpr int KV = S::KV, NG = S::KB / S::KV;
    if (lat_contig && bk.t < 2 * bc) {  // the always-zero H columns, written once per stage buffer
        const float z[KV] = {};
        const int b = bk.t >> 1, col = (bk.t & 1) ? 14 : 6;
        for (int st = 0; st < g.stages; ++st)
            for (int gg = 0; gg < NG; ++gg)
                for (int cc = 0; cc < 2; ++cc)
                    put_bv<MODE>(b_tile<MODE>(c, st, 1, 0, g.chunk), b_tile<MODE>(c, st, 1, S::NPART - 1, g.chunk),
                                 16 * b + col + cc, gg, z, lbo);
    }
    auto build_b = [&](int st, int kb) {
        unsigned char* P0 = b_tile<MODE>(c, st, 0, 0, g.chunk);
        unsigned char* P1 = b_tile<MODE>(c, st, 0, S::NPART - 1, g.chunk);
        unsigned char* H0 = b_tile<MODE>(c, st, 1, 0, g.chunk);
        unsigned char* H1 = b_tile<MODE>(c, st, 1, S::NPART - 1, g.chunk);
        if (!lat_contig) {  // one (member, latitude) item per thread, one bf16/tf32 value per store
            for (int it = bk.t; it < bc * S::KB; it += kTcThreads) {
                const int b = it / S::KB, k = it - b * S::KB;
                const int j = kb * S::KB + k;
                float2 e[5], o[5];
                const float2* F = g.four_out + (size_t)(b0 + b) * 5 * fs;  // m-contiguous
                for (int f = 0; f < 5; ++f) {
                    if (j < g.J2) {
                        const float2 gN = F[(size_t)f * fs + (size_t)j * (R + 1) + m];
                        const float2 gS = F[(size_t)f * fs + (size_t)(J - 1 - j) * (R + 1) + m];
                        e[f] = cadd(gN, gS);
                        o[f] = csub(gN, gS);
                    } else {
                        e[f] = o[f] = make_float2(0.f, 0.f);
                    }
                }
                const int pf[4] = {2, 0, 1, 4};  // C, A, B, E in four_out order A, B, C, D, E
                const int hf[3] = {3, 1, 0};     // D, B, A
                for (int col = 0; col < 16; ++col) {
                    const int comp = col & 7, cpar = col >> 3;
                    const float2* src = cpar ? o : e;
                    const float2 zp = src[pf[comp >> 1]];
                    const float vP = (comp & 1) ? zp.y : zp.x;
                    float vH = 0.f;
                    if (comp < 6) {
                        const float2 zh = src[hf[comp >> 1]];
                        vH = (comp & 1) ? zh.y : zh.x;
                    }
                    put_b<MODE>(P0, P1, 16 * b + col, k, vP, lbo);
                    put_b<MODE>(H0, H1, 16 * b + col, k, vH, lbo);
                }
            }
            return;
        }
        for (int it = bk.t; it < bc * 5 * NG; it += kTcThreads) {
            const int gg = it % NG, q = it / NG;
            const int f = q % 5, b = q / 5;
            const int j0 = kb * S::KB + gg * KV;
            const float2* F = g.four_out + (size_t)(b0 + b) * 5 * fs + (size_t)f * fs + fx.at(0, m);
            float2 gN[KV], gS[KV];
            if (j0 + KV <= g.J2) {
                // north j0 .. j0 + KV - 1 and south J - j0 - KV .. J - 1 - j0 (reversed)
                const float4* pn = reinterpret_cast<const float4*>(F + j0);
                const float4* ps = reinterpret_cast<const float4*>(F + (J - j0 - KV));
#pragma unroll
                for (int v = 0; v < KV / 2; ++v) {
                    const float4 a = pn[v], z = ps[v];
                    gN[2 * v] = make_float2(a.x, a.y);
                    gN[2 * v + 1] = make_float2(a.z, a.w);
                    gS[KV - 1 - 2 * v] = make_float2(z.x, z.y);
                    gS[KV - 2 - 2 * v] = make_float2(z.z, z.w);
                }
            } else {
#pragma unroll
                for (int v = 0; v < KV; ++v) {
                    const int j = j0 + v;
                    gN[v] = j < g.J2 ? F[j] : make_float2(0.f, 0.f);
                    gS[v] = j < g.J2 ? F[J - 1 - j] : make_float2(0.f, 0.f);
                }
            }
            float er[KV], ei[KV], orr[KV], oi[KV];
#pragma unroll
            for (int v = 0; v < KV; ++v) {
                const float2 e = cadd(gN[v], gS[v]), o = csub(gN[v], gS[v]);
                er[v] = e.x;
                ei[v] = e.y;
                orr[v] = o.x;
                oi[v] = o.y;
            }
            // four_out fields A, B, C, D, E -> (group, first column): A: P 2, H 4; B: P 4, H 2;
            // C: P 0; D: H 0; E: P 6
            const int cP = f == 0 ? 2 : f == 1 ? 4 : f == 2 ? 0 : f == 4 ? 6 : -1;
            const int cH = f == 0 ? 4 : f == 1 ? 2 : f == 3 ? 0 : -1;
#pragma unroll
            for (int grp = 0; grp < 2; ++grp) {
                const int c0 = grp == 0 ? cP : cH;
                if (c0 < 0) continue;
                unsigned char* t0 = grp == 0 ? P0 : H0;
                unsigned char* t1 = grp == 0 ? P1 : H1;
                const int r = 16 * b + c0;
                put_bv<MODE>(t0, t1, r, gg, er, lbo);
                put_bv<MODE>(t0, t1, r + 1, gg, ei, lbo);
                put_bv<MODE>(t0, t1, r + 8, gg, orr, lbo);
                put_bv<MODE>(t0, t1, r + 9, gg, oi, lbo);
            }
        }
    };
    const bool ok = k_loop<MODE>(bk, c, nkb, g.stages, g.chunk, tmem, N, idesc_for<MODE>(N), g.err, build_b, load_a);
    const int warp = bk.t >> 5, lane = bk.t & 31;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * warp) << 16);
    const int k = t * kTileRows + 32 * warp + lane;
    for (int b = 0; b < bc; ++b) {
        float vP[16], vH[16];
        tmem_ld16(lane_base + 16 * b, vP);
        tmem_ld16(lane_base + N + 16 * b, vH);
        if (!ok || k >= nm) continue;
        const bool par = k & 1;
        float P8[8], H8[8];  // C, A, B, E at this row's parity; D, B, A at the opposite one
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            P8[i] = par ? vP[8 + i] : vP[i];
            H8[i] = par ? vH[i] : vH[8 + i];
        }
        const float2 sC{P8[0], P8[1]}, sA{P8[2], P8[3]}, sB{P8[4], P8[5]}, sE{P8[6], P8[7]};
        const float2 hD{H8[0], H8[1]}, hB{H8[2], H8[3]}, hA{H8[4], H8[5]};
        const int n = m + k;
        // the nonlinear part from the float32 sums, combined in float32 (its
        // rounding is far below the operands' split-BF16 / TF32 rounding)
        double2 f0, f1, f2;
        fe_rows(sC, sA, sB, sE, hD, hB, hA, (float)m, g.ia_f, n, f0, f1, f2);
        // the Coriolis part, exactly in float64 (grid products carry no f)
        coriolis_add(g.state + (size_t)(b0 + b) * g.state_ms, g.cor, g.nc, R, m, n, off, g.two_omega, f1, f2);
        if (m == 0) f0.y = f1.y = f2.y = 0.0;
        double2* FE = g.FE + (size_t)(b0 + b) * g.fe_ms;
        FE[off + k] = f0;
        FE[g.nc + off + k] = f1;
        FE[2 * g.nc + off + k] = f2;
    }
    cta_release(bk, c, tmem, ncols);
}

// ------------------------------------------------ analysis, warp-specialised
// For batched launches (latitude-contiguous input, up to 8 members per CTA):
// 256 threads, persistent over the (m, 128 degrees) tiles bk.idx.x,
// bk.idx.x + bk.dim.x, ...  Warpgroup 0 (threads 0..127) builds the B
// operand of each K block while thread 0 issues the block's TMA loads and
// MMAs into one of two accumulator buffers in tensor memory (the tile's
// parity) and, after the tile's last block, commits to acc_full[buffer].
// Warpgroup 1 (threads 128..255) waits for acc_full, reads the accumulators
// (warp w reads lanes 32 (w % 4) .. 32 (w % 4) + 31), runs the epilogue of
// k_tc_anal and arrives on acc_empty[buffer]; thread 0 waits for that before
// the first MMA into the buffer two tiles later.  The epilogue of one tile
// thus runs while the next tile is loaded, built and multiplied.  Warpgroup
// 0 synchronises on named barrier 1 and checks the abort flag only after it,
// so its threads never diverge around the barrier; every wait is bounded.
// (Named barrier 1 in the kernel; in the persistent kernel, Blk::bar2.)
constexpr int kWsThreads = 256;

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// named barrier bk.bar2 over the producer warpgroup (threads 0..127 of the block)
__device__ __forceinline__ void producer_sync(const Blk& bk) {
    asm volatile("bar.sync %0, 128;" ::"r"(bk.bar2) : "memory");
}

template <int MODE>
__device__ __forceinline__ void b_tc_anal_ws(const Blk& bk, const Maps& maps, const TcArgs& g) {
    using S = Shape<MODE>;
    const int b0 = bk.idx.y * g.chunk;
    const int bc = min(g.chunk, g.members - b0);
    const int N = 16 * bc;
    const int R = g.R;
    const int nkb = (g.J2p + S::KB - 1) / S::KB;
    const int stages = g.stages;
    const uint32_t ncols = tmem_cols_for(4 * N);  // two accumulator buffers of 2N columns
    const Cta c = cta_setup<MODE>(bk, g.chunk, stages, ncols);
    uint64_t* acc_full = reinterpret_cast<uint64_t*>(c.smem + stages * c.stage_sz + 64);
    uint64_t* acc_empty = acc_full + 2;
    if (bk.t == 0) {
        mbar_init(sa(&acc_full[0]), 1);
        mbar_init(sa(&acc_full[1]), 1);
        mbar_init(sa(&acc_empty[0]), 4);  // one arrival per epilogue warp
        mbar_init(sa(&acc_empty[1]), 4);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    bk.sync();
    const uint32_t tmem = *c.tslot;
    const uint32_t lbo = lbo_for(N);
    const uint32_t idesc = idesc_for<MODE>(N);
    const int J = 2 * g.J2;
    const size_t fs = (size_t)J * (R + 1);
    constexpr int KV = S::KV, NG = S::KB / S::KV;
    const int warp = bk.t >> 5, lane = bk.t & 31;
    bool ok = true;
    // thread 0's TMA loads not yet waited for (stages 0, 1) and last committed K block
    int pend0 = -1, pend1 = -1, q_commit = -1;
    pdl_wait();
    if (bk.t < 128) {
        // ------------------------------------------------ producer warpgroup
        if (bk.t < 2 * bc) {  // the always-zero H columns, written once per stage buffer
            const float z[KV] = {};
            const int b = bk.t >> 1, col = (bk.t & 1) ? 14 : 6;
            for (int st = 0; st < stages; ++st)
                for (int gg = 0; gg < NG; ++gg)
                    for (int cc = 0; cc < 2; ++cc)
                        put_bv<MODE>(b_tile<MODE>(c, st, 1, 0, g.chunk), b_tile<MODE>(c, st, 1, S::NPART - 1, g.chunk),
                                     16 * b + col + cc, gg, z, lbo);
        }
        int q = 0, tcount = 0;
        for (int tile = bk.idx.x; tile < g.n_tiles; tile += bk.dim.x, ++tcount) {
            const int2 tl = g.tiles[tile];
            const int m = tl.x, t = tl.y;
            const int row = m * (R + 1) - m * (m - 1) / 2 + t * kTileRows;
            const int buf = tcount & 1;
            for (int kb = 0; kb < nkb; ++kb, ++q) {
                const int st = q % stages;
                // the MMAs that last read this stage must have completed
                if (q >= stages && !mbar_wait(sa(&c.bars[kMaxStages + st]), (uint32_t)(q / stages - 1) & 1)) {
                    atomicExch(g.err, kErrMmaTimeout);
                    *c.abort = 1;
                }
                if (bk.t == 0) {
                    mbar_expect_tx(sa(&c.bars[st]), (uint32_t)(S::NT * kTileBytes));
                    for (int i = 0; i < S::NT; ++i)
                        tma_load_2d(sa(a_tile<MODE>(c, st, i)), &maps.m[i], kb * S::KB, row, sa(&c.bars[st]));
                    if (st == 0) pend0 = q;
                    else pend1 = q;
                }
                unsigned char* P0 = b_tile<MODE>(c, st, 0, 0, g.chunk);
                unsigned char* P1 = b_tile<MODE>(c, st, 0, S::NPART - 1, g.chunk);
                unsigned char* H0 = b_tile<MODE>(c, st, 1, 0, g.chunk);
                unsigned char* H1 = b_tile<MODE>(c, st, 1, S::NPART - 1, g.chunk);
                for (int it = bk.t; it < bc * 5 * NG; it += 128) {
                    const int gg = it % NG, qq = it / NG;
                    const int f = qq % 5, b = qq / 5;
                    const int j0 = kb * S::KB + gg * KV;
                    const float2* F = g.four_out + (size_t)(b0 + b) * 5 * fs + (size_t)f * fs + (size_t)m * J;
                    float2 gN[KV], gS[KV];
                    if (j0 + KV <= g.J2) {
                        const float4* pn = reinterpret_cast<const float4*>(F + j0);
                        const float4* ps = reinterpret_cast<const float4*>(F + (J - j0 - KV));
#pragma unroll
                        for (int v = 0; v < KV / 2; ++v) {
                            const float4 a = pn[v], z = ps[v];
                            gN[2 * v] = make_float2(a.x, a.y);
                            gN[2 * v + 1] = make_float2(a.z, a.w);
                            gS[KV - 1 - 2 * v] = make_float2(z.x, z.y);
                            gS[KV - 2 - 2 * v] = make_float2(z.z, z.w);
                        }
                    } else {
#pragma unroll
                        for (int v = 0; v < KV; ++v) {
                            const int j = j0 + v;
                            gN[v] = j < g.J2 ? F[j] : make_float2(0.f, 0.f);
                            gS[v] = j < g.J2 ? F[J - 1 - j] : make_float2(0.f, 0.f);
                        }
                    }
                    float er[KV], ei[KV], orr[KV], oi[KV];
#pragma unroll
                    for (int v = 0; v < KV; ++v) {
                        const float2 e = cadd(gN[v], gS[v]), o = csub(gN[v], gS[v]);
                        er[v] = e.x;
                        ei[v] = e.y;
                        orr[v] = o.x;
                        oi[v] = o.y;
                    }
                    const int cP = f == 0 ? 2 : f == 1 ? 4 : f == 2 ? 0 : f == 4 ? 6 : -1;
                    const int cH = f == 0 ? 4 : f == 1 ? 2 : f == 3 ? 0 : -1;
#pragma unroll
                    for (int grp = 0; grp < 2; ++grp) {
                        const int c0 = grp == 0 ? cP : cH;
                        if (c0 < 0) continue;
                        unsigned char* t0 = grp == 0 ? P0 : H0;
                        unsigned char* t1 = grp == 0 ? P1 : H1;
                        const int r = 16 * b + c0;
                        put_bv<MODE>(t0, t1, r, gg, er, lbo);
                        put_bv<MODE>(t0, t1, r + 1, gg, ei, lbo);
                        put_bv<MODE>(t0, t1, r + 8, gg, orr, lbo);
                        put_bv<MODE>(t0, t1, r + 9, gg, oi, lbo);
                    }
                }
                fence_async_smem();
                tc_fence_before();
                producer_sync(bk);
                tc_fence_after();
                if (*c.abort) {  // read after the barrier: the same value in every producer thread
                    ok = false;
                    break;
                }
                if (bk.t == 0) {
                    // before the tile's first MMA: the epilogue of the tile two back has drained the buffer
                    if (kb == 0 && tcount >= 2 &&
                        !mbar_wait(sa(&acc_empty[buf]), (uint32_t)(tcount / 2 - 1) & 1)) {
                        atomicExch(g.err, kErrMmaTimeout);
                        *c.abort = 1;
                    } else if (!mbar_wait(sa(&c.bars[st]), (uint32_t)(q / stages) & 1)) {
                        atomicExch(g.err, kErrTmaTimeout);
                        *c.abort = 1;
                    } else {
                        if (st == 0) pend0 = -1;
                        else pend1 = -1;
                        tc_fence_after();
                        mma_block<MODE>(c, st, g.chunk, tmem + (uint32_t)(buf * 2 * N), N, idesc, kb == 0);
                        mma_commit(sa(&c.bars[kMaxStages + st]));
                        if (kb == nkb - 1) mma_commit(sa(&acc_full[buf]));
                        q_commit = q;
                    }
                }
            }
            if (!ok) break;
        }
        if (bk.t == 0 && (!ok || *c.abort)) {
            // a wait gave up: wait (bounded) for this CTA's loads and MMAs in flight
            if (pend0 >= 0) mbar_wait(sa(&c.bars[0]), (uint32_t)(pend0 / stages) & 1);
            if (pend1 >= 0) mbar_wait(sa(&c.bars[1]), (uint32_t)(pend1 / stages) & 1);
            if (q_commit >= 0)
                mbar_wait(sa(&c.bars[kMaxStages + q_commit % stages]), (uint32_t)(q_commit / stages) & 1);
        }
    } else {
        // ------------------------------------------------ epilogue warpgroup
        const uint32_t lane_rows = (uint32_t)(32 * (warp & 3)) << 16;
        int tcount = 0;
        for (int tile = bk.idx.x; tile < g.n_tiles; tile += bk.dim.x, ++tcount) {
            const int buf = tcount & 1;
            const int2 tl = g.tiles[tile];
            const int m = tl.x, t = tl.y;
            const int nm = R + 1 - m;
            const int off = m * (R + 1) - m * (m - 1) / 2;
            const int k = t * kTileRows + 32 * (warp & 3) + lane;
            // the first member's Coriolis operands, loaded while the tile's MMAs run
            CorIn cn{};
            if (k < nm) cn = coriolis_load(g.state + (size_t)b0 * g.state_ms, g.cor, g.nc, R, m, m + k, off);
            if (!mbar_wait(sa(&acc_full[buf]), (uint32_t)(tcount / 2) & 1)) {
                if (lane == 0) atomicExch(g.err, kErrMmaTimeout);
                *c.abort = 1;
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t base = tmem + lane_rows + (uint32_t)(buf * 2 * N);
            for (int b = 0; b < bc; ++b) {
                const CorIn cc = cn;
                if (k < nm && b + 1 < bc)
                    cn = coriolis_load(g.state + (size_t)(b0 + b + 1) * g.state_ms, g.cor, g.nc, R, m, m + k, off);
                float vP[16], vH[16];
                tmem_ld16(base + 16 * b, vP);
                tmem_ld16(base + N + 16 * b, vH);
                if (k >= nm) continue;
                const bool par = k & 1;
                float P8[8], H8[8];  // C, A, B, E at this row's parity; D, B, A at the opposite one
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    P8[i] = par ? vP[8 + i] : vP[i];
                    H8[i] = par ? vH[i] : vH[8 + i];
                }
                const float2 sC{P8[0], P8[1]}, sA{P8[2], P8[3]}, sB{P8[4], P8[5]}, sE{P8[6], P8[7]};
                const float2 hD{H8[0], H8[1]}, hB{H8[2], H8[3]}, hA{H8[4], H8[5]};
                const int n = m + k;
                double2 f0, f1, f2;
                fe_rows(sC, sA, sB, sE, hD, hB, hA, (float)m, g.ia_f, n, f0, f1, f2);
                coriolis_apply(cc, g.two_omega, f1, f2);
                if (m == 0) f0.y = f1.y = f2.y = 0.0;
                double2* FE = g.FE + (size_t)(b0 + b) * g.fe_ms;
                FE[off + k] = f0;
                FE[g.nc + off + k] = f1;
                FE[2 * g.nc + off + k] = f2;
            }
            // this warp's reads of the buffer are complete (tcgen05.wait::ld)
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(sa(&acc_empty[buf]));
        }
    }
    cta_release(bk, c, tmem, ncols, true);
}


// ------------------------------------------------------------------ kernels
template <int MODE>
__global__ void __launch_bounds__(kTcThreads, 1) k_tc_synth(const __grid_constant__ Maps maps,
                                                            const __grid_constant__ TcArgs g) {
    extern __shared__ unsigned char smem_tc[];
    b_tc_synth<MODE>(hw_blk(smem_tc), maps, g);
}
template <int MODE>
__global__ void __launch_bounds__(kTcThreads, 1) k_tc_anal(const __grid_constant__ Maps maps,
                                                           const __grid_constant__ TcArgs g) {
    extern __shared__ unsigned char smem_tc[];
    b_tc_anal<MODE>(hw_blk(smem_tc), maps, g);
}
template <int MODE>
__global__ void __launch_bounds__(kWsThreads, 1) k_tc_anal_ws(const __grid_constant__ Maps maps,
                                                              const __grid_constant__ TcArgs g) {
    extern __shared__ unsigned char smem_tc[];
    b_tc_anal_ws<MODE>(hw_blk(smem_tc), maps, g);
}

}  // namespace tc
}  // namespace mlsdc
