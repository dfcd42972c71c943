// Mixed-precision explicit right-hand side.  The Legendre sums and the
// longitude FFTs run in float32 (float32 FMAs on the CUDA cores for
// MLSDC_FP32; tcgen05 tensor cores for MLSDC_TF32 / MLSDC_BF16X3, see
// legendre_tc.cu); the state arrives in float64 and F_E leaves in float64,
// with the final combination (div, curl, n(n+1)/a^2 E) done in float64.
// F_E = L_F + N is evaluated as the exact float64 spectral Coriolis part
// (coriolis_linear) plus the nonlinear products through the transforms, so
// the reduced-precision error scales with the nonlinear terms (f is about ten
// times the vorticity) instead of the full (zeta + f) V flux.
// The float32 tables are rounded on the device from the float64 master tables
// that sh_plan computes on the host.
#include <algorithm>

#include "complex.cuh"
#include "convert.cuh"
#include "internal.h"
#include "rhs_kernels.cuh"

namespace mlsdc {

__global__ void k_round_f32(const double* __restrict__ x, float* __restrict__ y, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        y[i] = (float)x[i];
}

__global__ void k_round_c32(const double2* __restrict__ x, float2* __restrict__ y, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        y[i] = make_float2((float)x[i].x, (float)x[i].y);
}

mlsdc_status tc_init(sh_plan_t p);   // legendre_tc.cu
mlsdc_status tc_config(sh_plan_t p, int stage, int* chunk, int* stages, int* ws);
mlsdc_status tc_set_config(sh_plan_t p, int stage, int chunk, int stages, int ws);
mlsdc_status wait_selftest(int timeout_ms, int* code);
void tc_free(sh_plan_t p);
mlsdc_status tc_synth(sh_plan_t p, const double* state, double a, RhsBatch b, cudaStream_t st);
mlsdc_status tc_anal(sh_plan_t p, double a, double* FE, const double* state, double two_omega, RhsBatch b,
                     FourStride fo, cudaStream_t st);

constexpr int kStageAuto = 0, kStageTc = 1;

// each kernel's recorded arguments are its body's (persistent.cu)
MLSDC_SAME_PACK((k_synth_rhs<float, false>), (b_synth_rhs<float, false>));
MLSDC_SAME_PACK((k_synth_rhs<float, true>), (b_synth_rhs<float, true>));
MLSDC_SAME_PACK((k_synth_rhs<double, false>), (b_synth_rhs<double, false>));
MLSDC_SAME_PACK((k_grid_rhs<float, 1>), (b_grid_rhs<float, 1>));
MLSDC_SAME_PACK(k_anal_rhs<float>, b_anal_rhs<float>);
MLSDC_SAME_PACK(k_anal_rhs<double>, b_anal_rhs<double>);

// Which kernel a Legendre stage of a tensor-core plan runs for a launch of
// `members` states.  The rule is the outcome of timing both kernels on GB300
// for R = 21, 42, 85, 170 and 1..48 members: the tcgen05 analysis wins from
// R = 85 up, the tcgen05 synthesis only at R = 170 with 8 or more members
// (its 16 columns per member leave a single member's MMA mostly idle and the
// B operand costs more to stage than the CUDA-core sums).  A fixed rule keeps
// results reproducible run to run; the CUDA-core kernels use float32
// operands, at least as accurate as split-BF16 or TF32.
bool stage_uses_tc(const sh_plan_s* p, int stage, int members) {
    const int mode = stage == 0 ? p->mp.synth_mode : p->mp.anal_mode;
    if (mode != kStageAuto) return mode == kStageTc;
    return stage == 0 ? (p->R >= 128 && members >= 8) : p->R >= 64;
}

// Whether a float32 synthesis launch of `members` states streams its tables
// by TMA (synth_boxes(R) boxes of 32 rows per work item, all resident in
// shared memory) or reads them with plain loads.  The TMA form takes one
// table latency per work item instead of one per unrolled group of degrees,
// but its shared memory (8 KB per box) limits the CTAs per SM, so it pays for
// few boxes, and for three boxes only with few members (many members give the
// plain loads enough CTAs to hide their latency).
bool synth_uses_tma(const sh_plan_s* p, int members) {
    const MPTables& t = p->mp;
    if (!t.syn_tma || t.syn_tma_mode == 2) return false;
    if (t.syn_tma_mode == 1) return true;
    const int boxes = synth_boxes(p->R);
    return boxes <= 2 || (boxes <= 3 && members <= 4);
}

mlsdc_status mp_init(sh_plan_t p) {
    MPTables& t = p->mp;
    const size_t ntab = (size_t)p->nc * p->J2;
    const size_t nfour = (size_t)p->J * (p->R + 1);
    auto alloc = [&](void** ptr, size_t bytes) -> bool {
        if (cudaMalloc(ptr, bytes) != cudaSuccess) return false;
        p->bytes += (int64_t)bytes;
        return true;
    };
    bool ok = alloc((void**)&t.P32, ntab * sizeof(float)) && alloc((void**)&t.H32, ntab * sizeof(float)) &&
              alloc((void**)&t.tw32, (p->I / 2) * sizeof(float2)) &&
              alloc((void**)&t.stab32, (p->I / 2) * sizeof(float2)) &&
              alloc((void**)&t.four_in, 4 * nfour * p->max_members * sizeof(float2)) &&
              alloc((void**)&t.four_out, 5 * nfour * p->max_members * sizeof(float2)) &&
              alloc((void**)&t.lat32, (size_t)4 * p->J * sizeof(float)) &&
              alloc((void**)&t.invnn32, (size_t)(p->R + 1) * sizeof(float));
    if (!ok) {
        set_error("cudaMalloc (mixed-precision tables)", cudaGetLastError());
        return MLSDC_ERR_ALLOC;
    }
    k_round_f32<<<1024, 256>>>(p->d_P, t.P32, ntab);
    k_round_f32<<<1024, 256>>>(p->d_H, t.H32, ntab);
    k_round_c32<<<8, 256>>>(p->d_tw, t.tw32, p->I / 2);
    k_stage_twiddles<float2><<<1, 256>>>(t.stab32, t.tw32, p->I / 2, p->logI - 1, p->I);
    k_round_f32<<<8, 256>>>(p->d_lat, t.lat32, (size_t)4 * p->J);
    k_round_f32<<<8, 256>>>(p->d_invnn, t.invnn32, (size_t)(p->R + 1));
    MLSDC_LAUNCHED("k_round_f32");
    MLSDC_CUDA(cudaDeviceSynchronize());
    // the synthesis can stream its tables by TMA where the row pitch allows (J2 a multiple of 4 floats)
    MLSDC_CUDA(cudaMalloc((void**)&t.d_err, sizeof(int)));
    MLSDC_CUDA(cudaMemset(t.d_err, 0, sizeof(int)));
    const uint32_t bw = (uint32_t)std::min(32, p->J2);
    t.syn_tma = p->J2 % 4 == 0 &&
                make_rows_map_f32(&t.syn_maps.P, t.P32, (uint64_t)p->J2, (uint64_t)p->nc, bw, kSynBoxRows) &&
                make_rows_map_f32(&t.syn_maps.H, t.H32, (uint64_t)p->J2, (uint64_t)p->nc, bw, kSynBoxRows);
    mlsdc_status rs = raise_smem_limit((const void*)k_synth_rhs<float, false>, synth_smem<float>(p->R));
    if (rs == MLSDC_OK && t.syn_tma)
        rs = raise_smem_limit((const void*)k_synth_rhs<float, true>, synth_tma_smem(p->R));
    if (rs == MLSDC_OK) rs = raise_smem_limit((const void*)k_grid_rhs<float, 1>, grid_smem<float>(p->I));
    if (rs == MLSDC_OK) rs = raise_smem_limit((const void*)k_grid_rhs<float, 2>, grid_smem<float>(p->I, 2));
    if (rs != MLSDC_OK) return rs;
    if (p->precision == MLSDC_TF32 || p->precision == MLSDC_BF16X3) return tc_init(p);
    return MLSDC_OK;
}

void mp_free(sh_plan_t p) {
    MPTables& t = p->mp;
    tc_free(p);
    cudaFree(t.P32);
    cudaFree(t.H32);
    cudaFree(t.tw32);
    cudaFree(t.stab32);
    cudaFree(t.four_in);
    cudaFree(t.four_out);
    cudaFree(t.lat32);
    cudaFree(t.invnn32);
    cudaFree(t.d_err);
    t = MPTables();
}

mlsdc_status rhs_explicit_mp(sh_plan_t p, const swe_params* prm, const double* state, double* FE, cudaStream_t st,
                             int64_t* launches, int stage, RhsBatch b) {
    const int R = p->R;
    MPTables& t = p->mp;
    if (b.members < 1 || b.members > p->max_members) return MLSDC_ERR_INVALID;
    const bool tc = p->precision == MLSDC_TF32 || p->precision == MLSDC_BF16X3;
    const size_t fs = (size_t)p->J * (R + 1);
    const MemberStrides ms{b.state_ms, 4 * fs, 5 * fs, b.fe_ms};
    const FourStride fo = four_out_layout(p->J, R, b.members >= kLatContigMembers);
    mlsdc_status s;
    // A level whose FFT grid (one CTA per latitude and member) is at most
    // 128 CTAs -- the coarse level of a single-member step -- runs every
    // stage as a fraction of one wave: its synthesis and FFT kernels are
    // then launched with programmatic serialisation too, their CTAs waiting
    // on the SMs the predecessor leaves free.  Measured on the split-BF16
    // step (150-step runs, one box): 1070 -> 1087 (synthesis), 1088 (FFT),
    // 1101 steps/s (both); the synthesis at T170 as well (684 CTAs) 972,
    // the FFT at both levels 994: there the successor's early CTAs take SMs
    // the predecessor's later CTAs still need.
    const bool small_level = (size_t)p->J * b.members <= 128;
    if (stage == 0 || stage < 0) {
        PdlScope pdl(small_level);
        if (tc && stage_uses_tc(p, 0, b.members)) {
            if ((s = tc_synth(p, state, prm->a, b, st)) != MLSDC_OK) return s;
        } else {
            const bool tma = synth_uses_tma(p, b.members);
            const dim3 grid(p->n_synth, b.members), block(32 * kSynthWarps);
            const double na2 = -prm->a * prm->a, ia = 1.0 / prm->a;
            if (tma) {
                MLSDC_LAUNCH("k_synth_rhs<float, tma>",
                             launch_b(Body::SynthF32Tma, 0, 0, k_synth_rhs<float, true>, grid, block,
                                      synth_tma_smem(R), st, t.syn_maps, t.d_err, (const double2*)state,
                                      (const float*)t.P32, (const float*)t.H32, (const float*)t.invnn32,
                                      (const Chunk*)p->d_synth, R, p->J2, p->nc, na2, ia, t.four_in, ms));
            } else {
                MLSDC_LAUNCH("k_synth_rhs<float>",
                             launch_b(Body::SynthF32, 0, 0, k_synth_rhs<float, false>, grid, block,
                                      synth_smem<float>(R), st, t.syn_maps, (int*)nullptr, (const double2*)state,
                                      (const float*)t.P32, (const float*)t.H32, (const float*)t.invnn32,
                                      (const Chunk*)p->d_synth, R, p->J2, p->nc, na2, ia, t.four_in, ms));
            }
        }
    }
    if (stage == 1 || stage < 0) {
        PdlScope pdl(small_level);
        if (fo.sj == 1) {  // latitude-contiguous output: two adjacent latitudes per CTA
            MLSDC_LAUNCH("k_grid_rhs<float, 2>",
                         launch_b(Body::GridF32x2, 0, 0, k_grid_rhs<float, 2>, dim3(p->J / 2, b.members), dim3(256),
                                  grid_smem<float>(p->I, 2), st, (const float2*)t.four_in, t.four_out,
                                  (const float*)t.lat32, (const float2*)t.tw32, (const float2*)t.stab32, R, p->I, p->logI, p->J, 0.0, ms, fo));
        } else {
            MLSDC_LAUNCH("k_grid_rhs<float, 1>",
                         launch_b(Body::GridF32x1, 0, 0, k_grid_rhs<float, 1>, dim3(p->J, b.members), dim3(256), grid_smem<float>(p->I), st,
                                  (const float2*)t.four_in, t.four_out, (const float*)t.lat32,
                                  (const float2*)t.tw32, (const float2*)t.stab32, R, p->I, p->logI, p->J, 0.0, ms, fo));
        }
    }
    if (stage == 2 || stage < 0) {
        if (tc && stage_uses_tc(p, 2, b.members)) {
            PdlScope pdl(true);  // its set-up and first table tiles overlap the FFT kernel's tail
            if ((s = tc_anal(p, prm->a, FE, state, 2.0 * prm->omega, b, fo, st)) != MLSDC_OK) return s;
        } else {
            MLSDC_LAUNCH("k_anal_rhs<float>",
                         launch_b(Body::AnalF32, 0, anal_smem_bytes<float>(), k_anal_rhs<float>, dim3(p->n_anal, b.members), dim3(32 * anal_warps(p->J2)), 0, st,
                                  (const float2*)t.four_out, (const float*)t.P32, (const float*)t.H32,
                                  (const Chunk*)p->d_anal, R, p->J2, p->nc, 1.0 / prm->a,
                                  (double2*)FE, (const double2*)state, 2.0 * prm->omega, (const double*)p->d_cor, ms,
                                  fo));
        }
    }
    if (launches) *launches += stage < 0 ? 3 : 1;
    return MLSDC_OK;
}

// The integer-pipe conversion of convert.cuh next to the hardware one,
// element by element (mlsdc_selftest_convert).
__global__ void k_convert_selftest(const float* __restrict__ f_in, int n, double* __restrict__ d_ours,
                                   double* __restrict__ d_hw) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        d_ours[i] = f64_of(f_in[i]);
        d_hw[i] = (double)f_in[i];
    }
}

// The float32 synthesis's error word (0, or kErrTmaTimeout).
mlsdc_status mp_error(sh_plan_t p, int* code) {
    *code = 0;
    if (!p->mp.d_err) return MLSDC_OK;
    MLSDC_CUDA(cudaMemcpy(code, p->mp.d_err, sizeof(int), cudaMemcpyDeviceToHost));
    return MLSDC_OK;
}

}  // namespace mlsdc

extern "C" mlsdc_status sh_plan_stage_kernels(sh_plan_t p, int members, int* synth_tc, int* anal_tc) {
    if (!p || members < 1) return MLSDC_ERR_INVALID;
    const bool tc = p->precision == MLSDC_TF32 || p->precision == MLSDC_BF16X3;
    if (synth_tc) *synth_tc = tc && mlsdc::stage_uses_tc(p, 0, members) ? 1 : 0;
    if (anal_tc) *anal_tc = tc && mlsdc::stage_uses_tc(p, 2, members) ? 1 : 0;
    return MLSDC_OK;
}

extern "C" mlsdc_status sh_plan_tc_config(sh_plan_t p, int stage, int* members_per_cta, int* stages,
                                          int* warp_specialised) {
    if (!p) return MLSDC_ERR_INVALID;
    return mlsdc::tc_config(p, stage, members_per_cta, stages, warp_specialised);
}

extern "C" mlsdc_status mlsdc_selftest_wait_timeout(int timeout_ms, int* code) {
    if (!code || timeout_ms < 1 || timeout_ms > 2000) return MLSDC_ERR_INVALID;
    return mlsdc::wait_selftest(timeout_ms, code);
}

extern "C" mlsdc_status sh_plan_set_tc_config(sh_plan_t p, int stage, int members_per_cta, int stages,
                                              int warp_specialised) {
    if (!p || !(p->precision == MLSDC_TF32 || p->precision == MLSDC_BF16X3)) return MLSDC_ERR_INVALID;
    return mlsdc::tc_set_config(p, stage, members_per_cta, stages, warp_specialised);
}

extern "C" mlsdc_status mlsdc_selftest_convert(const float* f_in, int n, double* d_ours, double* d_hw,
                                              void* stream) {
    if (!f_in || !d_ours || !d_hw || n < 1) return MLSDC_ERR_INVALID;
    mlsdc::k_convert_selftest<<<std::min(1024, (n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(f_in, n, d_ours,
                                                                                                d_hw);
    MLSDC_LAUNCHED("k_convert_selftest");
    return MLSDC_OK;
}

extern "C" mlsdc_status sh_plan_set_synth_tma(sh_plan_t p, int mode) {
    if (!p || p->precision == MLSDC_FP64 || mode < 0 || mode > 2) return MLSDC_ERR_INVALID;
    p->mp.syn_tma_mode = mode;
    return MLSDC_OK;
}

extern "C" mlsdc_status sh_plan_set_stage_kernels(sh_plan_t p, int synth_mode, int anal_mode) {
    if (!p || !(p->precision == MLSDC_TF32 || p->precision == MLSDC_BF16X3)) return MLSDC_ERR_INVALID;
    if (synth_mode < 0 || synth_mode > 2 || anal_mode < 0 || anal_mode > 2) return MLSDC_ERR_INVALID;
    p->mp.synth_mode = synth_mode;
    p->mp.anal_mode = anal_mode;
    return MLSDC_OK;
}
