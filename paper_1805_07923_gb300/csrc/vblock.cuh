// Virtual thread blocks: every stage kernel of a step is written as a body
// that takes its block index, thread index, barrier and shared memory from a
// Blk instead of the hardware registers.  A kernel launched on its own
// passes the hardware values (hw_blk; after inlining the code is that of a
// plain kernel); the persistent ensemble kernel (persistent.cu) runs the same
// bodies for virtual blocks it takes from a phase's work list, several side
// by side in one CTA, each on its own slice of threads, named barrier and
// shared memory.
//
// The launches of a step are turned into such work lists by recording them:
// while a Recorder is installed on the calling thread, launch_b stores the
// body, the grid and the packed arguments of a launch instead of launching.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstring>
#include <type_traits>
#include <utility>
#include <vector>

namespace mlsdc {

struct Blk {
    uint3 idx, dim;      // block index and grid size
    unsigned t, nt;      // thread index in the block, threads per block (1-D blocks)
    unsigned bar;        // 0: the CTA's barrier; otherwise named barrier `bar` over nt threads
    unsigned bar2;       // a second named barrier the body may use for a subset of its threads
    unsigned char* smem; // the block's dynamic shared memory
    bool persist;        // inside the persistent kernel (no tensor-memory permit release)
    __device__ __forceinline__ void sync() const {
        if (bar == 0)
            __syncthreads();
        else
            asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(nt) : "memory");
    }
};

__device__ __forceinline__ Blk hw_blk(unsigned char* smem) {
    Blk b;
    b.idx = blockIdx;
    b.dim = gridDim;
    b.t = threadIdx.x;
    b.nt = blockDim.x;
    b.bar = 0;
    b.bar2 = 1;
    b.smem = smem;
    b.persist = false;
    return b;
}

// The bodies the persistent kernel can run (one per kernel and template
// instance).  Body::Count is the number of entries.
enum class Body : int {
    SynthF32,
    SynthF64,
    GridF32x1,
    GridF32x2,
    GridF64x1,
    AnalF32,
    AnalF64,
    TcSynthTf32,
    TcSynthBf16,
    TcAnalTf32,
    TcAnalBf16,
    TcAnalWsTf32,
    TcAnalWsBf16,
    ImplicitRhs,
    SweepNode,
    SweepNode0_2,
    SweepNode0_3,
    SweepNode0_4,
    SweepNode0_5,
    SweepNode0_6,
    SweepNode0_7,
    SweepNode0_8,
    SweepNodeS,
    Broadcast,
    Restrict,
    FasTau,
    Interp,
    PadAdd,
    Copy2D,
    SynthF32Tma,
    Count
};

// Kernel arguments packed back to back in declaration order (each member at
// its type's alignment), the layout host and device agree on.
template <class... T>
struct Pack {};
template <class H, class... T>
struct Pack<H, T...> {
    H h;
    Pack<T...> t;
};

template <class... K>
struct PackFill;
template <>
struct PackFill<> {
    static void fill(Pack<>&) {}
};
template <class H, class... T>
struct PackFill<H, T...> {
    template <class A, class... As>
    static void fill(Pack<H, T...>& p, A&& a, As&&... as) {
        p.h = H(std::forward<A>(a));
        PackFill<T...>::fill(p.t, std::forward<As>(as)...);
    }
};

template <class... K, class... A>
inline void fill_pack(Pack<K...>& p, A&&... a) {
    PackFill<K...>::fill(p, std::forward<A>(a)...);
}

// The pack type of a kernel's parameter list.
template <class F>
struct KernelPack;
template <class... K>
struct KernelPack<void (*)(K...)> {
    using type = Pack<std::decay_t<K>...>;
};

// The pack type of a body's parameter list after its Blk (references and
// const dropped): the same as its kernel's KernelPack, which launch_b records.
template <class F>
struct BodyPack;
template <class... K>
struct BodyPack<void (*)(const Blk&, K...)> {
    using type = Pack<std::decay_t<K>...>;
};

#define MLSDC_SAME_PACK(K, B) \
    static_assert(std::is_same<KernelPack<decltype(&K)>::type, BodyPack<decltype(&B)>::type>::value, #K)

// Call f(b, a_1, ..., a_n) with the members of a pack (by reference, so a
// body taking `const T&` reads the pack's copy in place).
template <class F, class... Done>
__device__ __forceinline__ void apply_pack(F& f, const Blk& b, const Pack<>&, const Done&... done) {
    f(b, done...);
}
template <class F, class H, class... T, class... Done>
__device__ __forceinline__ void apply_pack(F& f, const Blk& b, const Pack<H, T...>& p, const Done&... done) {
    apply_pack(f, b, p.t, done..., p.h);
}

// One recorded launch.
struct RecLaunch {
    Body body;
    dim3 grid, block;
    size_t smem;        // dynamic shared memory the body needs (bytes)
    int tmem_cols;      // tensor-memory columns one block allocates (0: none)
    int op, sub;        // the step operation it belongs to and its place among that operation's launches
    std::vector<unsigned char> args;
};

struct Recorder {
    std::vector<RecLaunch> recs;
    int op = 0, sub = 0;
    bool refused = false;  // a launch of a kernel without a body was attempted
    void begin_op(int o) {
        op = o;
        sub = 0;
    }
};

// The recorder installed on this thread (null: launches run).
Recorder*& active_recorder();

template <class Kern, class... Args>
inline void record_launch(Recorder* r, Body body, int tmem_cols, size_t smem, Kern kernel, dim3 grid, dim3 block,
                          Args&&... args) {
    using P = typename KernelPack<Kern>::type;
    (void)kernel;
    P p;
    std::memset((void*)&p, 0, sizeof(P));
    fill_pack(p, std::forward<Args>(args)...);
    RecLaunch L;
    L.body = body;
    L.grid = grid;
    L.block = block;
    L.smem = smem;
    L.tmem_cols = tmem_cols;
    L.op = r->op;
    L.sub = r->sub++;
    L.args.resize(sizeof(P));
    std::memcpy(L.args.data(), (const void*)&p, sizeof(P));
    r->recs.push_back(std::move(L));
}

}  // namespace mlsdc
