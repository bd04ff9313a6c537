// tma.cuh -- column pass with its tile staged in shared memory by the tensor
// memory accelerator (TMA), for the diffraction half of the split-step march
// (arXiv 2306.15678, Eq. 2).
//
// A column tile is C columns of n points: n rows of C * 8 bytes (complex64),
// every row in another DRAM page.  Moved by per-thread loads and stores, each
// warp request touches 32/C cache lines and the SM's load/store unit becomes
// the bottleneck of the pass.  Here one thread moves the tile with 2D bulk
// tensor copies of 256-row boxes (cp.async.bulk.tensor) into a row-major
// [n][C] stage, completion counted in bytes on an mbarrier; the threads then
// read their column values from shared memory, transform them exactly as
// k_col_pass does (bit for bit), write the results back to the stage, and the
// same thread stores the stage with bulk tensor copies.  The stage aliases the
// transform lines: it is read before the first exchange and written after the
// last one.
//
// Waits are bounded by a %globaltimer deadline: on expiry the block records
// bit 1 (NLSE_ETIMEOUT) in the status word, waits once more, bounded, for the
// copy it started, and returns without touching the field.  If that second
// wait runs out too, the copy may still be in flight into shared memory that
// a later block can be given: the block also sets bit 2, which the host
// reports as NLSE_ETIMEOUT as well and which means that the output of this
// launch and of every later kernel on the stream is not to be trusted.  Bulk tensor
// copies need a 128-byte aligned shared-memory address; dynamic shared memory
// is only guaranteed 16 bytes, so the launch adds kTmaAlignPad bytes and the
// kernel aligns the base at run time.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.cuh"

namespace nlse {

constexpr int kTmaBoxRows = 256;                   // rows per bulk copy (largest box dimension)
constexpr long long kTmaTimeoutNs = 1000000000LL;  // 1 s per wait
constexpr int kTmaAlign = 128;                     // shared-memory alignment of a bulk tensor copy
constexpr int kTmaAlignPad = kTmaAlign;            // extra dynamic shared memory for aligning

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ long long global_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// true when the phase completed before the deadline
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > kTmaTimeoutNs) return false;
    return true;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, int x, int y, int z, const void* src) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];"
                 ::"l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(src))
                 : "memory");
}
// commit the block's bulk stores and wait until they have read their source:
// the shared memory may then be released (the writes complete on their own,
// before the kernel does)
__device__ __forceinline__ void tma_store_commit_and_wait_read() {
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
// make this thread's generic-proxy shared-memory writes visible to bulk copies
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// order this thread's global-memory accesses of the generic proxy (including
// data it acquired from other threads) with its bulk copies, both ways
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}
// commit the block's bulk stores and wait until their writes are complete
__device__ __forceinline__ void tma_store_commit_and_wait() {
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// The staged tile exists where the column is a whole number of boxes (a box
// holds kTmaBoxRows row pairs of the state layout, see sidx) and the stage fits
// in the transform lines it aliases.  A box row -- the two values of a row pair
// in each of the C columns -- is 16 C (complex64) or 32 C (complex128) bytes.
template <typename T, int N, int C> __host__ __device__ constexpr bool col_tma_valid() {
    return N % (2 * kTmaBoxRows) == 0 && N <= line_stride<T, N, C>() && threads_per_line<T, N>() * C <= 1024 &&
           line_stride<T, N, C>() * C * (int)sizeof(typename vec2<T>::type) + kTmaAlignPad <= 232448;
}

// Column pass with the tile staged by bulk tensor copies.  mload / mstore
// describe src / dst (state layout) as 3D arrays of n/2 row pairs x n columns x
// 4 words (the real and imaginary parts of the pair's two values; the copies
// move bits); a box holds kTmaBoxRows row pairs of C columns and lands in the
// stage as [pair][column][2 values].  Thread layout and arithmetic are
// col_tile's.
// status may be null.  extra_tx (a test hook, 0 in use) makes block 0 expect
// that many bytes more than its copies bring, so that its wait runs out.
template <typename T, int N, int C>
__global__ void __launch_bounds__(threads_per_line<T, N>() * C, min_blocks<threads_per_line<T, N>() * C>())
k_col_pass_tma(const __grid_constant__ CUtensorMap mload, const __grid_constant__ CUtensorMap mstore,
               const typename tab_of<T>::type* __restrict__ tw, const typename tab_of<T>::type* __restrict__ px,
               const typename tab_of<T>::type* __restrict__ py, typename tab_of<T>::type rot,
               int* __restrict__ status, uint32_t extra_tx) {
    using V = typename vec2<T>::type;
    constexpr int E = elems<T, N>(), TL = threads_per_line<T, N>();
    constexpr int LS = line_stride<T, N, C>(), BOXES = N / (2 * kTmaBoxRows);
    constexpr uint32_t BYTES = (uint32_t)(N * C * sizeof(V));
    static_assert(col_tma_valid<T, N, C>(), "staged column tile");
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ uint64_t bar;
    __shared__ int s_fail;
    const uint32_t pad = (kTmaAlign - (smem_u32(smraw) & (kTmaAlign - 1))) & (kTmaAlign - 1);
    V* smem = reinterpret_cast<V*>(smraw + pad);
    V* stage = smem;  // [N/2][C][2], aliased by the transform lines once read
    const int col0 = blockIdx.x * C;
    // stage index of (y, c): [y/2][c][y mod 2]
    auto st = [](int y, int c) { return C == 1 ? y : ((y >> 1) * C + c) * 2 + (y & 1); };
    pdl_trigger();
    pdl_wait();
    if (threadIdx.x == 0) {
        s_fail = 0;
        mbar_init(&bar, 1);
        mbar_expect_tx(&bar, BYTES + (blockIdx.x == 0 ? extra_tx : 0u));
#pragma unroll 1
        for (int b = 0; b < BOXES; ++b)
            tma_load_3d(stage + b * kTmaBoxRows * C * 2, &mload, 0, col0, b * kTmaBoxRows, &bar);
        if (!mbar_wait_bounded(&bar, 0)) {
            if (status) atomicOr(status, 2);
            // the copy still targets this block's memory: wait for it once more
            if (!mbar_wait_bounded(&bar, 0) && status) atomicOr(status, 4);
            s_fail = 1;
        }
    }
    __syncthreads();
    if (s_fail) return;  // (uniform)
    const int c = threadIdx.x % C, j = threadIdx.x / C;
    const int col = col0 + c;
    V v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = stage[st(j + m * TL, c)];
    __syncthreads();  // the staged tile is consumed; the transforms reuse its memory
    V* sm = smem + c * LS;
#pragma unroll 1
    for (int half = 0; half < 2; ++half) {
        if (half == 1) conj_all(v);  // second round: B_y = conj(F_y(conj(.)))
        fft_stockham<V, N, E, false>(v, sm, tw, j);
        if (half == 0) {
            const auto pxc = tabmul(ldent(px + col), rot);
#pragma unroll
            for (int m = 0; m < E; ++m) v[m] = twmul<false>(twmul<false>(v[m], pxc), ldent(py + j + m * TL));
        }
    }
    conj_all(v);
#pragma unroll
    for (int m = 0; m < E; ++m) stage[st(j + m * TL, c)] = v[m];
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll 1
        for (int b = 0; b < BOXES; ++b)
            tma_store_3d(&mstore, 0, col0, b * kTmaBoxRows, stage + b * kTmaBoxRows * C * 2);
        tma_store_commit_and_wait_read();
    }
}

}  // namespace nlse
