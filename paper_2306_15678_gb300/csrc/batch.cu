// batch.cu -- many beams of different grid sizes marched together in one
// persistent launch (FP32), the data parallelism the paper's independent
// statistical realisations and test beams offer (Sec. 2 and Sec. 3.3).
//
// Work items are (step, pass, beam, tile), numbered step by step as [column
// tiles of every beam][row tiles of every beam]; blocks claim them in that
// order from one atomic counter.  A column tile of beam b at step s needs all
// row tiles of b at step s-1 done, a row tile needs all column tiles of b at
// step s: per-beam completion counters carry this.  Every item waits only on
// items numbered before it, and those were claimed by blocks that were
// running, so progress never depends on how many blocks are resident.  Waits
// are bounded by a deadline on %globaltimer; on expiry the block records
// NLSE_ETIMEOUT in the status word, raises an abort flag that stops every
// other block, and returns.
//
// Tile bodies are the per-pass kernels' own (row_tile32 / col_body32 of the
// pair engine, radix 16 or 8), with field accesses that bypass L1 because
// other SMs rewrite the fields during the launch, so a batched beam is
// bit-identical to the same beam marched alone at the same radix.  Column tiles
// of beams with n >= 512 are moved by bulk tensor copies (as the single grid's
// staged column pass does, one tensor map per beam in the workspace); the
// copies read rows that other blocks wrote with ordinary stores and write
// columns that other blocks read with ordinary loads, so the block orders the
// two proxies around them (fence.proxy.async) on both sides of the completion
// counters.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/nlse.h"
#include "dispatch32.cuh"
#include "host_detail.h"

namespace nlse {

constexpr int kBatchMinLog2 = 8, kBatchMaxLog2 = 12;  // n = 256 .. 4096
constexpr int kRotSteps = 1 << 20;  // steps covered by the per-step phase table

struct BatchBeam {
    float4* field;     // unit layout (pass32.cuh)
    const float2* px;  // kDitherP copies of n entries each (copy k mod kDitherP serves step k)
    const unsigned char* py;  // kDitherP copies of P_y and the cross-lane factors (py32_copy_bytes)
    const unsigned char* tw;  // kDither twiddle blocks (pass32.cuh: tw32_copy_bytes)
    const CUtensorMap* map;   // the field as n/2 row pairs x n columns x 4 words, boxes of one
                              // column x 256 row pairs (staged column tiles; null for n < 512)
    ScreenCoef<float> sc;
    int log2n;
    int col_tiles;
    int row_tiles;
    int pad;
};

struct BatchPlan {
    const BatchBeam* beams;
    const int* col_off;  // prefix sums of column tiles, nbeams + 1 entries
    const int* row_off;  // prefix sums of row tiles, nbeams + 1 entries
    int nbeams;
    int items_per_step;
    int nsteps;
    unsigned int* next;
    unsigned int* done_col;
    unsigned int* done_row;
    int* status;
    int* abort;
    const long long* step_base;  // steps taken before this launch
    const float2* rot;           // rot[k] = exp(i theta_{k+1}) in FP32 (k: 0-based global step)
    long long timeout_ns;
    long long skip_item;  // test hook: this item never reports completion (-1: none)
    int staged;           // column tiles of beams with n >= 512 staged by bulk tensor copies
};

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// row pairs / columns per tile for a block of THREADS threads at radix E
template <int THREADS, int E, int N> __host__ __device__ constexpr int tile_pairs() {
    return THREADS / p_tpl<N, E>();
}
template <int THREADS, int E, int N> __host__ __device__ constexpr int tile_cols() {
    return THREADS / p_col_tpl<N, E>();
}
template <int THREADS, int E, int N> __host__ __device__ constexpr int batch_row_smem() {
    return pr::pair_line_stride<N, p_e<N, E>(), tile_pairs<THREADS, E, N>()>() * tile_pairs<THREADS, E, N>() * 16;
}
template <int THREADS, int E, int N> __host__ __device__ constexpr bool batch_supported() {
    return p_tpl<N, E>() <= THREADS && p_col_tpl<N, E>() <= THREADS && tile_pairs<THREADS, E, N>() <= N / 2 &&
           tile_cols<THREADS, E, N>() <= N && batch_row_smem<THREADS, E, N>() <= kMaxSmem - kTmaAlignPad &&
           p_col_smem<N, E, tile_cols<THREADS, E, N>()>() <= kMaxSmem - kTmaAlignPad;
}
// column tiles staged by bulk tensor copies: whole 256-row-pair boxes (n >= 512)
template <int THREADS, int E, int N> __host__ __device__ constexpr bool batch_staged() {
    if constexpr (batch_supported<THREADS, E, N>())
        return p_col_tma_valid<N, E, tile_cols<THREADS, E, N>()>();
    else
        return false;
}
template <int THREADS, int E, int N> __host__ __device__ constexpr int batch_smem() {
    if constexpr (batch_supported<THREADS, E, N>())
        return std::max(batch_row_smem<THREADS, E, N>(), p_col_smem<N, E, tile_cols<THREADS, E, N>()>());
    else
        return 0;
}
template <int THREADS, int E> constexpr int batch_smem_max() {
    return std::max({batch_smem<THREADS, E, 256>(), batch_smem<THREADS, E, 512>(), batch_smem<THREADS, E, 1024>(),
                     batch_smem<THREADS, E, 2048>(), batch_smem<THREADS, E, 4096>()}) +
           kTmaAlignPad;
}

// Per-block state of the staged column tiles: the block's mbarrier, its phase
// (kept by thread 0) and a failure flag for the whole block.
struct StageState {
    uint64_t* bar;
    uint32_t parity;
    int* fail;
};

// One staged column tile (beam with n >= 512): thread 0 orders the rows other
// blocks wrote (acquired through the completion counter) before its bulk
// copies, moves the C columns into their transform lines with one box of 256
// row pairs per copy and waits for them, bounded; every thread transforms its
// column exactly as col_tile32 does; thread 0 stores the lines back with bulk
// copies and waits until those writes are complete, so that the completion
// signal that follows covers them.  On a wait that runs out the block records
// bit 1 (and bit 2 if the copies may still be in flight), raises the abort
// flag and returns false without touching the field.
template <int THREADS, int E, int N>
__device__ __forceinline__ bool batch_col_staged(const BatchBeam& bm, int tile, const unsigned char* twb,
                                                 const float2* px, const float4* py, float2 rot, C2* smem,
                                                 StageState& st, const BatchPlan& plan) {
    constexpr int L = N / 2, EE = p_e<L, E>(), T = p_col_tpl<N, E>(), C = tile_cols<THREADS, E, N>();
    constexpr int LS = pr::pair_line_stride<L, EE, C>(), BOXES = L / kTmaBoxRows;
    constexpr uint32_t BYTES = (uint32_t)(C * L * 16);
    const int col0 = tile * C;
    if (threadIdx.x == 0) {
        int fail = 0;
        fence_proxy_async_global();  // the acquired rows, before the copies read them
        fence_proxy_async_smem();    // this block's earlier use of the lines, before the copies write them
        mbar_expect_tx(st.bar, BYTES);
#pragma unroll 1
        for (int c = 0; c < C; ++c)
#pragma unroll 1
            for (int b = 0; b < BOXES; ++b)
                tma_load_3d(smem + c * LS + b * kTmaBoxRows, bm.map, 0, col0 + c, b * kTmaBoxRows, st.bar);
        if (!mbar_wait_bounded(st.bar, st.parity)) {
            atomicOr(plan.status, 2);
            atomicExch(plan.abort, 1);
            if (!mbar_wait_bounded(st.bar, st.parity)) atomicOr(plan.status, 4);
            fail = 1;
        }
        st.parity ^= 1u;
        *st.fail = fail;
    }
    __syncthreads();
    if (*st.fail) return false;  // (uniform)
    const int c = (int)threadIdx.x / T, j = (int)threadIdx.x % T;
    C2* line = smem + c * LS;
    C2 v[EE];
#pragma unroll
    for (int m = 0; m < EE; ++m) v[m] = line[j + m * T];
    __syncthreads();  // the staged tile is consumed; the transforms reuse its memory
    col_body32<N, E>(v, line, twb, px, py, rot, col0 + c, j);
#pragma unroll
    for (int m = 0; m < EE; ++m) line[j + m * T] = v[m];
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll 1
        for (int cc = 0; cc < C; ++cc)
#pragma unroll 1
            for (int b = 0; b < BOXES; ++b)
                tma_store_3d(bm.map, 0, col0 + cc, b * kTmaBoxRows, smem + cc * LS + b * kTmaBoxRows);
        tma_store_commit_and_wait();
        fence_proxy_async_global();  // the copies' writes, before the completion signal
    }
    return true;
}

// one tile of global step k with the step's table copy, as a single grid applies
// it; false if a staged copy failed (the item then reports no completion)
template <int THREADS, int E, int N>
__device__ __forceinline__ bool batch_tile(const BatchBeam& bm, bool col, int tile, long long k, float2 rot,
                                           C2* smem, StageState& st, const BatchPlan& plan) {
    if constexpr (batch_supported<THREADS, E, N>()) {
        const int d = (int)(k & (kDither - 1)), dp = (int)(k & (kDitherP - 1));
        const unsigned char* twb = bm.tw + (size_t)d * tw32_copy_bytes(N);
        if (col) {
            constexpr int C = tile_cols<THREADS, E, N>();
            const float2* px = bm.px + (size_t)dp * N;
            const float4* py = reinterpret_cast<const float4*>(bm.py + (size_t)dp * py32_copy_bytes(N));
            if constexpr (batch_staged<THREADS, E, N>()) {
                if (plan.staged) return batch_col_staged<THREADS, E, N>(bm, tile, twb, px, py, rot, smem, st, plan);
            }
            col_tile32<N, E, C, UnitCG>(bm.field, bm.field, twb, px, py, rot, tile * C, smem);
        } else {
            constexpr int RP = tile_pairs<THREADS, E, N>();
            float ts = 0.f, tm = 0.f;
            row_tile32<N, E, RP, false, UnitCG>(bm.field, bm.field, twb, bm.sc, tile * RP, smem, ts, tm);
        }
    }
    return true;
}

// registers: 128 per thread at radix 16, about 85 at radix 8 (the column
// body's propagator and cross-lane factors on top of the transform)
template <int THREADS, int E>
__global__ void __launch_bounds__(THREADS, p_col_min_blocks<THREADS, E>()) k_batch_march(BatchPlan plan) {
    extern __shared__ __align__(16) unsigned char smraw[];
    // 128-byte aligned base: the staged column tiles land there by bulk copies
    const uint32_t pad = (kTmaAlign - (smem_u32(smraw) & (kTmaAlign - 1))) & (kTmaAlign - 1);
    C2* smem = reinterpret_cast<C2*>(smraw + pad);
    __shared__ int s_item_step, s_item_beam, s_item_tile, s_item_col, s_stop, s_fail;
    __shared__ float2 s_rot;
    __shared__ long long s_k;
    __shared__ uint64_t s_bar;
    if (threadIdx.x == 0 && plan.staged) mbar_init(&s_bar, 1);
    StageState st{&s_bar, 0u, &s_fail};
    const long long total = (long long)plan.items_per_step * plan.nsteps;
    const int col_total = plan.col_off[plan.nbeams];
    for (;;) {
        if (threadIdx.x == 0) {
            int stop = 0;
            long long i = -1;
            if (*(volatile int*)plan.abort) stop = 1;
            else i = (long long)atomicAdd(plan.next, 1u);
            if (!stop && i >= total) stop = 1;
            if (!stop) {
                const int s = (int)(i / plan.items_per_step), r = (int)(i % plan.items_per_step);
                const bool col = r < col_total;
                const int* off = col ? plan.col_off : plan.row_off;
                const int rr = col ? r : r - col_total;
                int lo = 0, hi = plan.nbeams - 1;  // last beam with off[b] <= rr
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (off[mid] <= rr) lo = mid; else hi = mid - 1;
                }
                const BatchBeam& bm = plan.beams[lo];
                // dependency: all row tiles of step s-1 (column items) or all
                // column tiles of step s (row items) of this beam
                const unsigned int need = col ? (unsigned int)s * bm.row_tiles : (unsigned int)(s + 1) * bm.col_tiles;
                const unsigned int* ctr = col ? plan.done_row + lo : plan.done_col + lo;
                if (need > 0 && ld_acquire(ctr) < need) {
                    const long long t0 = global_ns();
                    while (ld_acquire(ctr) < need) {
                        if (*(volatile int*)plan.abort) { stop = 1; break; }
                        if (global_ns() - t0 > plan.timeout_ns) {
                            atomicOr(plan.status, 2);  // bit 1: a bounded wait ran out
                            atomicExch(plan.abort, 1);
                            stop = 1;
                            break;
                        }
                        __nanosleep(100);
                    }
                }
                const long long k = *plan.step_base + s;  // global step index
                s_k = k;
                s_rot = plan.rot[k];  // this step's global phase
                s_item_step = (int)(i & 0x7fffffff);
                s_item_beam = lo;
                s_item_tile = rr - off[lo];
                s_item_col = col;
            }
            s_stop = stop;
        }
        __syncthreads();
        if (s_stop) return;
        const int b = s_item_beam, tile = s_item_tile;
        const bool col = s_item_col != 0;
        const long long item = s_item_step;
        const float2 rot = s_rot;
        const long long k = s_k;
        const BatchBeam bm = plan.beams[b];
        bool ok = true;
        switch (bm.log2n) {
            case 8: ok = batch_tile<THREADS, E, 256>(bm, col, tile, k, rot, smem, st, plan); break;
            case 9: ok = batch_tile<THREADS, E, 512>(bm, col, tile, k, rot, smem, st, plan); break;
            case 10: ok = batch_tile<THREADS, E, 1024>(bm, col, tile, k, rot, smem, st, plan); break;
            case 11: ok = batch_tile<THREADS, E, 2048>(bm, col, tile, k, rot, smem, st, plan); break;
            case 12: ok = batch_tile<THREADS, E, 4096>(bm, col, tile, k, rot, smem, st, plan); break;
            default: break;
        }
        if (!ok) return;  // (uniform) the abort flag is raised
        __threadfence();  // this thread's tile stores, before the completion signal
        __syncthreads();
        if (threadIdx.x == 0 && item != plan.skip_item)
            atomicAdd(col ? plan.done_col + b : plan.done_row + b, 1u);
    }
}

__global__ void k_batch_advance(long long* step_base, int nsteps) { *step_base += nsteps; }

}  // namespace nlse

using namespace nlse;

namespace {

constexpr int kBatchChunk = 1 << 20;  // steps per persistent launch (keeps item indices below 2^31)

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }
int ilog2i(int n) {
    int k = 0;
    while ((1 << k) < n) ++k;
    return (1 << k) == n ? k : -1;
}

template <int THREADS, int E> int tiles_for(int log2n, bool col) {
    auto f = [&](auto nc) -> int {
        constexpr int N = decltype(nc)::value;
        if constexpr (batch_supported<THREADS, E, N>())
            return col ? N / tile_cols<THREADS, E, N>() : N / 2 / tile_pairs<THREADS, E, N>();
        else return 0;
    };
    switch (log2n) {
        case 8: return f(std::integral_constant<int, 256>{});
        case 9: return f(std::integral_constant<int, 512>{});
        case 10: return f(std::integral_constant<int, 1024>{});
        case 11: return f(std::integral_constant<int, 2048>{});
        case 12: return f(std::integral_constant<int, 4096>{});
    }
    return 0;
}

struct BLayout {
    std::vector<size_t> field, px, py;
    size_t tw[kBatchMaxLog2 + 1];
    size_t maps, beams, col_off, row_off, counters, step_base, rot, partials, readout, scratch, total;
};

BLayout blayout(int count, const nlse_params* ps) {
    BLayout L;
    size_t o = 0;
    L.field.resize(count);
    L.px.resize(count);
    L.py.resize(count);
    for (int b = 0; b < count; ++b) {
        L.field[b] = o; o = al256(o + (size_t)ps[b].n * ps[b].n * 8);
    }
    for (int b = 0; b < count; ++b) {
        L.px[b] = o; o = al256(o + (size_t)kDitherP * ps[b].n * 8);
        L.py[b] = o; o = al256(o + (size_t)kDitherP * py32_copy_bytes(ps[b].n));
    }
    int maxn = 0;
    for (int k = 0; k <= kBatchMaxLog2; ++k) L.tw[k] = 0;
    for (int b = 0; b < count; ++b) maxn = std::max(maxn, (int)ps[b].n);
    for (int k = kBatchMinLog2; k <= kBatchMaxLog2; ++k) {
        bool used = false;
        for (int b = 0; b < count; ++b) used |= ps[b].n == (1 << k);
        if (used) { L.tw[k] = o; o = al256(o + (size_t)kDither * tw32_copy_bytes(1 << k)); }
    }
    L.maps = o;      o = al256(o + sizeof(CUtensorMap) * count);  // 64-byte aligned each
    L.beams = o;     o = al256(o + sizeof(BatchBeam) * count);
    L.col_off = o;   o = al256(o + sizeof(int) * (count + 1));
    L.row_off = o;   o = al256(o + sizeof(int) * (count + 1));
    L.counters = o;  o = al256(o + sizeof(unsigned int) * (2 * count + 1) + 2 * sizeof(int));
    L.step_base = o; o = al256(o + sizeof(long long));
    L.rot = o;       o = al256(o + sizeof(float2) * (size_t)kRotSteps);
    L.partials = o;  o = al256(o + (size_t)maxn * 2 * sizeof(double));
    L.readout = o;   o = al256(o + 4 * sizeof(double) + sizeof(int));
    L.scratch = o;   o = al256(o + (size_t)maxn * maxn * 8);  // field staging for host readouts
    L.total = o;
    return L;
}

nlse_status bvalidate(int count, const nlse_params* ps) {
    if (count < 1 || !ps) return NLSE_EINVAL;
    for (int b = 0; b < count; ++b) {
        size_t bytes;
        nlse_status st = nlse_workspace_size(&ps[b], &bytes);
        if (st != NLSE_OK) return st;
        if (ps[b].precision != NLSE_FP32 || ps[b].scheme != NLSE_LIE) return NLSE_EUNSUPPORTED;
        const int k = ilog2i(ps[b].n);
        if (k < kBatchMinLog2 || k > kBatchMaxLog2) return NLSE_EUNSUPPORTED;
    }
    return NLSE_OK;
}

}  // namespace

struct nlse_batch {
    int count;
    std::vector<nlse_params> ps;
    std::vector<int> log2n, col_tiles, row_tiles;
    cudaStream_t stream;
    unsigned char* ws;
    BLayout lay;
    nlse_batch_tuning tune;
    int grid;
    int smem;
    int64_t steps;
    double theta;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    int graph_steps;
};

namespace {


template <int THREADS, int E> nlse_status plan_tiles(nlse_batch* B) {
    for (int b = 0; b < B->count; ++b) {
        const int tc = tiles_for<THREADS, E>(B->log2n[b], true), tr = tiles_for<THREADS, E>(B->log2n[b], false);
        if (tc == 0 || tr == 0) return NLSE_EUNSUPPORTED;
        B->col_tiles[b] = tc;
        B->row_tiles[b] = tr;
    }
    B->smem = batch_smem_max<THREADS, E>();
    return NLSE_OK;
}

template <int THREADS, int E> nlse_status launch_batch(nlse_batch* B, int nsteps) {
    BatchPlan plan;
    unsigned char* ws = B->ws;
    unsigned int* ctr = reinterpret_cast<unsigned int*>(ws + B->lay.counters);
    plan.beams = reinterpret_cast<const BatchBeam*>(ws + B->lay.beams);
    plan.col_off = reinterpret_cast<const int*>(ws + B->lay.col_off);
    plan.row_off = reinterpret_cast<const int*>(ws + B->lay.row_off);
    plan.nbeams = B->count;
    int ct = 0, rt = 0;
    for (int b = 0; b < B->count; ++b) { ct += B->col_tiles[b]; rt += B->row_tiles[b]; }
    plan.items_per_step = ct + rt;
    plan.nsteps = nsteps;
    plan.next = ctr;
    plan.done_col = ctr + 1;
    plan.done_row = ctr + 1 + B->count;
    plan.status = reinterpret_cast<int*>(ctr + 1 + 2 * B->count);
    plan.abort = plan.status + 1;
    plan.step_base = reinterpret_cast<const long long*>(ws + B->lay.step_base);
    plan.rot = reinterpret_cast<const float2*>(ws + B->lay.rot);
    plan.timeout_ns = (long long)B->tune.timeout_ms * 1000000LL;
    plan.skip_item = B->tune.debug_skip_item;
    plan.staged = B->tune.per_thread_columns ? 0 : 1;
    // reset the work counter, the completion counters and the abort flag (not the status word)
    if (cudaMemsetAsync(ctr, 0, sizeof(unsigned int) * (1 + 2 * B->count), B->stream) != cudaSuccess)
        return NLSE_ECUDA;
    if (cudaMemsetAsync(plan.abort, 0, sizeof(int), B->stream) != cudaSuccess) return NLSE_ECUDA;
    k_batch_march<THREADS, E><<<B->grid, THREADS, B->smem, B->stream>>>(plan);
    if (cudaGetLastError() != cudaSuccess) return NLSE_ECUDA;
    k_batch_advance<<<1, 1, 0, B->stream>>>(reinterpret_cast<long long*>(ws + B->lay.step_base), nsteps);
    return cudaGetLastError() == cudaSuccess ? NLSE_OK : NLSE_ECUDA;
}

// the launch shapes: threads per block (128, 256, 512) x transform radix (16, 8;
// radix 8 at 256 and 512 threads)
template <typename F> nlse_status with_shape(const nlse_batch_tuning& t, F&& f) {
    if (t.threads == 512)
        return t.radix == 8 ? f(std::integral_constant<int, 512>{}, std::integral_constant<int, 8>{})
                            : f(std::integral_constant<int, 512>{}, std::integral_constant<int, 16>{});
    if (t.threads == 128)
        return t.radix == 8 ? NLSE_EUNSUPPORTED
                            : f(std::integral_constant<int, 128>{}, std::integral_constant<int, 16>{});
    return t.radix == 8 ? f(std::integral_constant<int, 256>{}, std::integral_constant<int, 8>{})
                        : f(std::integral_constant<int, 256>{}, std::integral_constant<int, 16>{});
}

nlse_status launch_any(nlse_batch* B, int nsteps) {
    return with_shape(B->tune, [&](auto th, auto e) {
        return launch_batch<decltype(th)::value, decltype(e)::value>(B, nsteps);
    });
}

void advance_host(nlse_batch* B, int nsteps) {
    for (int s = 0; s < nsteps; ++s) {
        double th = 0.0;  // the angle step B->steps + s turns the fields by
        detail::rot_step_f32(B->steps + s, &th);
        B->theta = std::fmod(B->theta + th, 6.283185307179586476925286766559);
    }
    B->steps += nsteps;
}

template <int THREADS, int E> nlse_status configure(nlse_batch* B) {
    auto kern = k_batch_march<THREADS, E>;
    if (B->smem > 48 * 1024 &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, B->smem) != cudaSuccess)
        return NLSE_ECUDA;
    // as much of the SM's unified memory as shared memory as the blocks can use
    if (cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared) !=
        cudaSuccess)
        return NLSE_ECUDA;
    int dev = 0, sms = 0, occ = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return NLSE_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return NLSE_ECUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, THREADS, B->smem) != cudaSuccess)
        return NLSE_ECUDA;
    if (occ < 1) return NLSE_EUNSUPPORTED;
    const int per_sm = B->tune.ctas_per_sm > 0 ? std::min(B->tune.ctas_per_sm, occ) : occ;
    B->grid = sms * per_sm;
    return NLSE_OK;
}

}  // namespace

extern "C" {

nlse_status nlse_batch_workspace_size(int32_t count, const nlse_params* params, size_t* bytes) {
    if (!bytes) return NLSE_EINVAL;
    nlse_status st = bvalidate(count, params);
    if (st != NLSE_OK) return st;
    *bytes = blayout(count, params).total;
    return NLSE_OK;
}

nlse_status nlse_batch_create(int32_t count, const nlse_params* params, const nlse_batch_tuning* tuning,
                              void* cuda_stream, void* dev_workspace, size_t workspace_bytes,
                              nlse_batch** out) {
    if (!out || !dev_workspace) return NLSE_EINVAL;
    *out = nullptr;
    nlse_status st = bvalidate(count, params);
    if (st != NLSE_OK) return st;
    if (reinterpret_cast<uintptr_t>(dev_workspace) & 255) return NLSE_EINVAL;
    BLayout lay = blayout(count, params);
    if (workspace_bytes < lay.total) return NLSE_ENOMEM;
    nlse_batch_tuning tn = {256, 0, 2000, -1, 16, 0};
    if (tuning) tn = *tuning;
    if (tn.radix == 0) tn.radix = 16;
    if (tn.threads != 128 && tn.threads != 256 && tn.threads != 512) return NLSE_EINVAL;
    if (tn.radix != 16 && tn.radix != 8) return NLSE_EINVAL;
    if (tn.ctas_per_sm < 0 || tn.timeout_ms < 1) return NLSE_EINVAL;
    if (tn.per_thread_columns != 0 && tn.per_thread_columns != 1) return NLSE_EINVAL;
    nlse_batch* B = new (std::nothrow) nlse_batch();
    if (!B) return NLSE_ENOMEM;
    B->count = count;
    B->ps.assign(params, params + count);
    B->log2n.resize(count);
    B->col_tiles.resize(count);
    B->row_tiles.resize(count);
    for (int b = 0; b < count; ++b) B->log2n[b] = ilog2i(params[b].n);
    B->stream = static_cast<cudaStream_t>(cuda_stream);
    B->ws = static_cast<unsigned char*>(dev_workspace);
    B->lay = lay;
    B->tune = tn;
    st = with_shape(tn, [&](auto th, auto e) {
        constexpr int TH = decltype(th)::value, E = decltype(e)::value;
        nlse_status r = plan_tiles<TH, E>(B);
        return r == NLSE_OK ? configure<TH, E>(B) : r;
    });
    if (st != NLSE_OK) { delete B; return st; }
    // per-beam tables and descriptors (built with the single-grid code so that
    // a batched beam and the same beam alone use identical tables)
    std::vector<BatchBeam> desc(count);
    std::vector<CUtensorMap> maps(count);
    std::vector<int> coff(count + 1, 0), roff(count + 1, 0);
    bool tw_done[kBatchMaxLog2 + 1] = {};
    for (int b = 0; b < count; ++b) {
        // the same table construction as a single grid, so that a batched beam
        // and the same beam alone use identical tables; the twiddles depend on
        // the size only and are uploaded once per size
        const bool need_tw = !tw_done[B->log2n[b]];
        tw_done[B->log2n[b]] = true;
        st = detail::upload_tables_f32(&params[b], B->stream, B->ws + lay.px[b], B->ws + lay.py[b],
                                       need_tw ? B->ws + lay.tw[B->log2n[b]] : nullptr);
        if (st != NLSE_OK) { delete B; return st; }
        BatchBeam& d = desc[b];
        d.field = reinterpret_cast<float4*>(B->ws + lay.field[b]);
        d.px = reinterpret_cast<const float2*>(B->ws + lay.px[b]);
        d.py = B->ws + lay.py[b];
        d.tw = B->ws + lay.tw[B->log2n[b]];
        d.map = nullptr;
        if (params[b].n >= 2 * kTmaBoxRows) {
            if (encode_field_map(&maps[b], d.field, params[b].n, 4, 1) != cudaSuccess) {
                delete B;
                return NLSE_ECUDA;
            }
            d.map = reinterpret_cast<const CUtensorMap*>(B->ws + lay.maps) + b;
        }
        d.sc = detail::screen_coef_f32(&params[b]);
        d.log2n = B->log2n[b];
        d.col_tiles = B->col_tiles[b];
        d.row_tiles = B->row_tiles[b];
        d.pad = 0;
        coff[b + 1] = coff[b] + d.col_tiles;
        roff[b + 1] = roff[b] + d.row_tiles;
    }
    const long long zero = 0;
    std::vector<float2> rot(kRotSteps);
    for (int s = 0; s < kRotSteps; ++s) rot[s] = detail::rot_step_f32(s, nullptr);
    if (cudaMemcpyAsync(B->ws + lay.rot, rot.data(), sizeof(float2) * rot.size(), cudaMemcpyHostToDevice,
                        B->stream) != cudaSuccess ||
        cudaMemcpyAsync(B->ws + lay.beams, desc.data(), sizeof(BatchBeam) * count, cudaMemcpyHostToDevice,
                        B->stream) != cudaSuccess ||
        cudaMemcpyAsync(B->ws + lay.maps, maps.data(), sizeof(CUtensorMap) * count, cudaMemcpyHostToDevice,
                        B->stream) != cudaSuccess ||
        cudaMemcpyAsync(B->ws + lay.col_off, coff.data(), sizeof(int) * (count + 1), cudaMemcpyHostToDevice,
                        B->stream) != cudaSuccess ||
        cudaMemcpyAsync(B->ws + lay.row_off, roff.data(), sizeof(int) * (count + 1), cudaMemcpyHostToDevice,
                        B->stream) != cudaSuccess ||
        cudaMemcpyAsync(B->ws + lay.step_base, &zero, sizeof(zero), cudaMemcpyHostToDevice, B->stream) !=
            cudaSuccess ||
        cudaMemsetAsync(B->ws + lay.counters, 0, sizeof(unsigned int) * (2 * count + 1) + 2 * sizeof(int),
                        B->stream) != cudaSuccess ||
        cudaStreamSynchronize(B->stream) != cudaSuccess) {
        delete B;
        return NLSE_ECUDA;
    }
    *out = B;
    return NLSE_OK;
}

}  // extern "C"

namespace {
// twiddles of the one-off transforms of a beam (load prologue, readouts): copy 0, as a single grid uses
const float2* fixed_twiddles(const nlse_batch* B, int beam) {
    return reinterpret_cast<const float2*>(B->ws + B->lay.tw[B->log2n[beam]]);
}
}  // namespace

extern "C" {

nlse_status nlse_batch_load_field(nlse_batch* B, int32_t beam, const void* src, int src_on_device) {
    if (!B || !src || beam < 0 || beam >= B->count) return NLSE_EINVAL;
    if (B->steps != 0) return NLSE_ESTATE;  // all beams start from the same step
    const int n = B->ps[beam].n;
    float2* f = reinterpret_cast<float2*>(B->ws + B->lay.field[beam]);
    const float2* tw = fixed_twiddles(B, beam);
    const KernelSet<float>* ks = kernels_f32(B->log2n[beam]);
    cudaError_t e;
    if (src_on_device) {
        e = ks->row_forward((const float2*)src, f, tw, B->stream);
    } else {
        // staged in the scratch buffer: the state layout differs from the rows'
        float2* rows = reinterpret_cast<float2*>(B->ws + B->lay.scratch);
        e = cudaMemcpyAsync(rows, src, (size_t)n * n * 8, cudaMemcpyHostToDevice, B->stream);
        if (e == cudaSuccess) e = ks->row_forward(rows, f, tw, B->stream);
    }
    return e == cudaSuccess ? NLSE_OK : NLSE_ECUDA;
}

nlse_status nlse_batch_step(nlse_batch* B, int32_t nsteps) {
    if (!B || nsteps < 0) return NLSE_EINVAL;
    if (B->steps + nsteps > kRotSteps) return NLSE_EUNSUPPORTED;
    while (nsteps > 0) {
        const int chunk = std::min(nsteps, kBatchChunk);
        nlse_status st = launch_any(B, chunk);
        if (st != NLSE_OK) return st;
        advance_host(B, chunk);
        nsteps -= chunk;
    }
    return NLSE_OK;
}

nlse_status nlse_batch_capture(nlse_batch* B, int32_t nsteps) {
    if (!B || nsteps < 1 || nsteps > kBatchChunk) return NLSE_EINVAL;
    if (B->exec) { cudaGraphExecDestroy(B->exec); B->exec = nullptr; }
    if (B->graph) { cudaGraphDestroy(B->graph); B->graph = nullptr; }
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return NLSE_ECUDA;
    cudaStream_t saved = B->stream;
    B->stream = cs;
    nlse_status st = NLSE_OK;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) st = NLSE_ECUDA;
    if (st == NLSE_OK) st = launch_any(B, nsteps);
    cudaGraph_t graph = nullptr;
    if (cudaStreamEndCapture(cs, &graph) != cudaSuccess && st == NLSE_OK) st = NLSE_ECUDA;
    B->stream = saved;
    cudaStreamDestroy(cs);
    if (st != NLSE_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (cudaGraphInstantiate(&B->exec, graph, 0) != cudaSuccess) {
        cudaGraphDestroy(graph);
        return NLSE_ECUDA;
    }
    B->graph = graph;
    B->graph_steps = nsteps;
    return NLSE_OK;
}

nlse_status nlse_batch_replay(nlse_batch* B) {
    if (!B) return NLSE_EINVAL;
    if (!B->exec) return NLSE_ESTATE;
    if (B->steps + B->graph_steps > kRotSteps) return NLSE_EUNSUPPORTED;
    if (cudaGraphLaunch(B->exec, B->stream) != cudaSuccess) return NLSE_ECUDA;
    advance_host(B, B->graph_steps);
    return NLSE_OK;
}

nlse_status nlse_batch_status(nlse_batch* B) {
    if (!B) return NLSE_EINVAL;
    int word[2] = {0, 0};
    int* status = reinterpret_cast<int*>(B->ws + B->lay.counters + sizeof(unsigned int) * (1 + 2 * B->count));
    if (cudaMemcpyAsync(word, status, sizeof(word), cudaMemcpyDeviceToHost, B->stream) != cudaSuccess)
        return NLSE_ECUDA;
    if (cudaMemsetAsync(status, 0, sizeof(int), B->stream) != cudaSuccess) return NLSE_ECUDA;
    if (cudaStreamSynchronize(B->stream) != cudaSuccess) return NLSE_ECUDA;
    if (word[0] & 6) return NLSE_ETIMEOUT;  // bit 1: a wait ran out; bit 2: a copy may still be in flight
    return NLSE_OK;
}

nlse_status nlse_batch_steps_taken(nlse_batch* B, int64_t* steps) {
    if (!B || !steps) return NLSE_EINVAL;
    *steps = B->steps;
    return NLSE_OK;
}

nlse_status nlse_batch_read_field(nlse_batch* B, int32_t beam, void* dst, int dst_on_device) {
    if (!B || !dst || beam < 0 || beam >= B->count) return NLSE_EINVAL;
    const int n = B->ps[beam].n;
    const KernelSet<float>* ks = kernels_f32(B->log2n[beam]);
    float2* f = reinterpret_cast<float2*>(B->ws + B->lay.field[beam]);
    const float2* tw = fixed_twiddles(B, beam);
    double* partials = reinterpret_cast<double*>(B->ws + B->lay.partials);
    float2 unrot = make_float2((float)std::cos(B->theta), (float)(-std::sin(B->theta)));
    if (dst_on_device) {
        if (ks->readout(f, tw, (float2*)dst, nullptr, partials, unrot, B->stream) != cudaSuccess)
            return NLSE_ECUDA;
        return NLSE_OK;
    }
    float2* stage = reinterpret_cast<float2*>(B->ws + B->lay.scratch);
    if (ks->readout(f, tw, stage, nullptr, partials, unrot, B->stream) != cudaSuccess) return NLSE_ECUDA;
    if (cudaMemcpyAsync(dst, stage, (size_t)n * n * 8, cudaMemcpyDeviceToHost, B->stream) != cudaSuccess)
        return NLSE_ECUDA;
    return cudaStreamSynchronize(B->stream) == cudaSuccess ? NLSE_OK : NLSE_ECUDA;
}

nlse_status nlse_batch_power(nlse_batch* B, int32_t beam, double* watts) {
    if (!B || !watts || beam < 0 || beam >= B->count) return NLSE_EINVAL;
    const KernelSet<float>* ks = kernels_f32(B->log2n[beam]);
    float2* f = reinterpret_cast<float2*>(B->ws + B->lay.field[beam]);
    const float2* tw = fixed_twiddles(B, beam);
    double* partials = reinterpret_cast<double*>(B->ws + B->lay.partials);
    double* out = reinterpret_cast<double*>(B->ws + B->lay.readout);
    if (ks->readout(f, tw, nullptr, nullptr, partials, make_float2(1.f, 0.f), B->stream) != cudaSuccess)
        return NLSE_ECUDA;
    const double dx = B->ps[beam].L / B->ps[beam].n;
    if (detail::finalize(partials, ks->row_blocks, dx * dx, out, reinterpret_cast<int*>(out + 4), B->stream) !=
        cudaSuccess)
        return NLSE_ECUDA;
    double r[2];
    if (cudaMemcpyAsync(r, out, sizeof(r), cudaMemcpyDeviceToHost, B->stream) != cudaSuccess) return NLSE_ECUDA;
    if (cudaStreamSynchronize(B->stream) != cudaSuccess) return NLSE_ECUDA;
    *watts = r[0];
    return std::isfinite(r[0]) ? NLSE_OK : NLSE_ENONFINITE;
}

nlse_status nlse_batch_destroy(nlse_batch* B) {
    if (!B) return NLSE_EINVAL;
    cudaError_t e = cudaStreamSynchronize(B->stream);
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    delete B;
    return e == cudaSuccess ? NLSE_OK : NLSE_ECUDA;
}

}  // extern "C"
