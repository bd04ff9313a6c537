// hot_areas.cuh -- "hot areas" of the beam cross-section (arXiv 2306.15678,
// Sec. 3.3): the closed regions where the fluence w = |U|^2 reaches a cut-off
// w_p, counted as the connected components of the thresholded grid (4 edge
// neighbours, or 8 with the corners; the window is not periodic).
//
// Labelling in four launches over a row-major int32 label array:
//  1. runs:   one block per row labels each pixel with w >= w_p by the index
//             of the first pixel of its horizontal run (block max-scans of
//             run starts over coalesced chunks of the row), every other pixel
//             by -1;
//  2. merge:  the runs of neighbouring rows that touch are joined by a
//             concurrent union-find over the run starts: the larger of two
//             roots is linked under the smaller with atomicMin, and a union
//             that finds its root already linked retries from the new parent;
//  3. roots:  every run start finds its root, compresses its path and counts
//             itself when it is a root;
//  4. spread: every pixel takes the root of its run start.
// Links always point to smaller indices, so every walk ends, and the root of a
// region is its smallest run start, which is its smallest pixel index: the
// labels are unique and equal to a sequential flood fill's, whatever order the
// device joins the runs in.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace nlse {

constexpr int kHotUnionTries = 1 << 20;  // bound on the retries of one union (never reached)
constexpr int kHotStatusGaveUp = 1;      // bit of the per-call status word

// 1. runs: one block of blockDim = min(n, 256) threads per row, sweeping the
// row in chunks of blockDim consecutive pixels (coalesced); pixel (y, x) of the
// row-major input is w[(y n + x) stride] (stride 2 reads the real parts of a
// complex array).  A pixel starts a run when it is on and its left neighbour is
// not; its label is the last run start at or before it: a block max-scan of
// the starts within the chunk, carried over from the previous chunks.
template <typename T>
__global__ void __launch_bounds__(256) k_hot_runs(const T* __restrict__ w, int n, int stride, T wp,
                                                  int* __restrict__ label) {
    __shared__ int warp_last[8];
    __shared__ int carry_s;
    const int y = blockIdx.x;
    const T* row = w + (size_t)y * n * stride;
    int* lrow = label + (size_t)y * n;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned mask = blockDim.x >= 32 ? 0xffffffffu : (1u << blockDim.x) - 1u;
    int carry = -1;  // last run start before the chunk
    for (int x0 = 0; x0 < n; x0 += blockDim.x) {
        const int x = x0 + threadIdx.x;
        const bool on = row[(size_t)x * stride] >= wp;
        const bool left_on = x > 0 && row[(size_t)(x - 1) * stride] >= wp;
        int incl = on && !left_on ? x : -1;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(mask, incl, o);
            if (lane >= o) incl = max(incl, v);
        }
        if (lane == 31 || threadIdx.x == blockDim.x - 1) warp_last[warp] = incl;
        __syncthreads();
        int cur = max(carry, incl);
        for (int k = 0; k < warp; ++k) cur = max(cur, warp_last[k]);
        lrow[x] = on ? y * n + cur : -1;
        if (threadIdx.x == blockDim.x - 1) carry_s = cur;
        __syncthreads();
        carry = carry_s;
    }
}

// root of pixel i: follow the links (each to a smaller index) to a self-labelled
// run start; reads bypass L1 so that links made by other blocks are seen
__device__ __forceinline__ int hot_find(const int* label, int i) {
    for (;;) {
        const int p = __ldcg(&label[i]);
        if (p == i) return i;
        i = p;
    }
}

__device__ __forceinline__ void hot_union(int* label, int a, int b, int* status) {
    for (int t = 0; t < kHotUnionTries; ++t) {
        a = hot_find(label, a);
        b = hot_find(label, b);
        if (a == b) return;
        if (a > b) {
            const int s = a;
            a = b;
            b = s;
        }
        const int old = atomicMin(&label[b], a);
        if (old == b) return;  // b was still a root: it now hangs under a
        b = old;               // b was linked meanwhile: join a with b's parent instead
    }
    atomicOr(status, kHotStatusGaveUp);
}

// 2. merge: pixel i of rows 0..n-2 joins its run with the runs below it that it
// touches.  With 4 neighbours only the left end of each vertical overlap joins
// (its left neighbours are not both on); with 8, a pixel whose lower neighbour is
// off also joins the runs at its lower corners.
__global__ void __launch_bounds__(256) k_hot_merge(int* __restrict__ label, int n, int conn, int* __restrict__ status) {
    const int nn1 = (n - 1) * n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nn1; i += gridDim.x * blockDim.x) {
        if (__ldcg(&label[i]) < 0) continue;
        const int x = i & (n - 1);
        const bool down = __ldcg(&label[i + n]) >= 0;
        if (down) {
            if (!(x > 0 && __ldcg(&label[i - 1]) >= 0 && __ldcg(&label[i - 1 + n]) >= 0))
                hot_union(label, i, i + n, status);
        } else if (conn == 8) {
            if (x > 0 && __ldcg(&label[i + n - 1]) >= 0) hot_union(label, i, i + n - 1, status);
            if (x + 1 < n && __ldcg(&label[i + n + 1]) >= 0) hot_union(label, i, i + n + 1, status);
        }
    }
}

// 3. roots: the forest is fixed now; every run start finds its root, points
// every start on its path at it, and the roots are counted
__global__ void __launch_bounds__(256) k_hot_roots(int* __restrict__ label, int n, int* __restrict__ count) {
    const int nn = n * n;
    int local = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += gridDim.x * blockDim.x) {
        if (label[i] < 0 || ((i & (n - 1)) > 0 && label[i - 1] >= 0)) continue;  // not a run start
        const int r = hot_find(label, i);
        if (r == i) {
            ++local;
            continue;
        }
        for (int s = i; s != r;) {
            const int p = __ldcg(&label[s]);
            if (p != r) label[s] = r;
            s = p;
        }
    }
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(count, local);
}

// 4. spread: every pixel takes its run start's root
__global__ void __launch_bounds__(256) k_hot_spread(int* __restrict__ label, int nn) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += gridDim.x * blockDim.x) {
        const int s = label[i];
        if (s < 0) continue;
        const int r = __ldcg(&label[s]);
        if (r != s) label[i] = r;
    }
}

}  // namespace nlse
