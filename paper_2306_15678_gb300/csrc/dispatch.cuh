// dispatch.cuh -- host-side launchers of the march kernels for every supported
// grid size n = 2^k (8..8192) and precision, gathered into per-size tables.
#pragma once
#include <cuda_runtime.h>
#include <utility>

#include <cudaTypedefs.h>

#include "adjoint.cuh"
#include "kernels.cuh"
#include "tma.cuh"
#include "turbulence.cuh"

namespace nlse {

constexpr int kMaxSmem = 232448;  // 227 KB opt-in shared memory per block (sm_100/103)
// column-tile codes: a width of 1..16 columns per block, or'ed with kColTma
// for the variant that stages the tile with bulk tensor copies (tma.cuh), and
// in FP32 with kColR8 for the radix-8 column transform (8 elements per thread;
// radix 16 without it)
constexpr int kColTma = 0x100;
constexpr int kColR8 = 0x200;
// row-pass code: radix 16 with persistent blocks that stage each row pair by a
// bulk copy (pass32.cuh: k_row_pass32_pf), or'ed with the radix
constexpr int kRowStaged = 0x100;
constexpr int kColOptionCount = 20;
constexpr int kColOptions[kColOptionCount] = {
    1, 2, 4, 8, 16, kColTma | 1, kColTma | 2, kColTma | 4, kColTma | 8, kColTma | 16,
    kColR8 | 1, kColR8 | 2, kColR8 | 4, kColR8 | 8, kColR8 | 16,
    kColR8 | kColTma | 1, kColR8 | kColTma | 2, kColR8 | kColTma | 4, kColR8 | kColTma | 8, kColR8 | kColTma | 16};

template <typename T> struct KernelSet {
    using V = typename vec2<T>::type;
    using W = typename tab_of<T>::type;
    int n;
    int row_blocks;    // blocks (partials) of the readout and of the default-radix row pass
    int row_blocks8;   // blocks (partials) of the radix-8 row pass
    int adj_blocks;    // blocks (partials) of the loss seed and the backward row pass
    int col_mask;      // bit i set: column tile kColOptions[i] is instantiated
    int col_default;   // default column tile
    int row_radix_mask;     // bit 0: radix 16 available for the row pass, bit 1: radix 8,
                            // bit 2: radix 16 with staged persistent blocks (kRowStaged | 16)
    int row_radix_default;  // default radix of the row pass (16 or 8)
    // rad: row-pass code (16, 8 or kRowStaged | 16; FP64: 8); status: device
    // status word (bit 1: a bounded wait ran out), may be null; extra_tx: test
    // hook of the staged variant (0 in use)
    cudaError_t (*row_pass)(const V* src, V* dst, const W* tw, ScreenCoef<T> sc, double* partials,
                            bool diag, int rad, int* status, unsigned extra_tx, cudaStream_t s);
    // status: device status word (bit 1: a bounded wait ran out), may be null;
    // extra_tx: test hook of the staged variant (0 in use)
    cudaError_t (*col_pass)(const V* src, V* dst, const W* tw, const W* px, const W* py, W rot,
                            int cols, int* status, unsigned extra_tx, cudaStream_t s);
    cudaError_t (*row_forward)(const V* src, V* dst, const W* tw, cudaStream_t s);
    cudaError_t (*readout)(const V* state, const W* tw, V* field_out, T* flu_out, double* partials,
                           V unrot, cudaStream_t s);
    cudaError_t (*loss_seed)(const V* state, V* gam, const double* target, const W* tw,
                             double seed_scale, double* partials, cudaStream_t s);
    cudaError_t (*adj_row)(V* gam, const V* tn, const W* tw, AdjCoef<T> ac, double* acc, cudaStream_t s);
    // unnormalised 2D DFT (inverse: conjugate kernel) of a row-major array, in place
    cudaError_t (*dft2)(V* data, const W* tw, bool inverse, cudaStream_t s);
};

// Raise the dynamic shared-memory limit of one kernel once per device.  The
// record is per kernel (the template argument is the kernel itself).
template <auto Kernel> inline cudaError_t ensure_smem(int bytes) {
    static unsigned long long done = 0;
    if (bytes <= 48 * 1024) return cudaSuccess;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (done & bit) return cudaSuccess;
    e = cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done |= bit;
    return e;
}

// The same, and the preferred shared-memory carveout of the kernel set to the
// smallest share of the SM's unified L1/shared array that holds `blocks`
// resident blocks of `bytes` dynamic shared memory each: the rest stays L1
// cache, where the twiddle and propagator tables are read from.
template <auto Kernel> inline cudaError_t ensure_smem_carveout(int bytes, int blocks) {
    static unsigned long long done = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (done & bit) return cudaSuccess;
    if (bytes > 48 * 1024 &&
        (e = cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) != cudaSuccess)
        return e;
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, Kernel)) != cudaSuccess) return e;
    int per_sm = 0;
    if ((e = cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess)
        return e;
    // 1 KB per block is reserved by the system
    const long long need = (long long)blocks * ((long long)bytes + (long long)fa.sharedSizeBytes + 1024);
    int pct = per_sm > 0 ? (int)((need * 100 + per_sm - 1) / per_sm) : 100;
    pct = pct < 1 ? 1 : (pct > 100 ? 100 : pct);
    if ((e = cudaFuncSetAttribute(Kernel, cudaFuncAttributePreferredSharedMemoryCarveout, pct)) != cudaSuccess)
        return e;
    done |= bit;
    return cudaSuccess;
}

template <typename T, int N> constexpr int row_smem_bytes() {
    return line_stride<T, N, rows_per_block<T, N>()>() * rows_per_block<T, N>() *
           (int)sizeof(typename vec2<T>::type);
}
template <typename T, int N, int C> constexpr int col_smem_bytes() {
    return line_stride<T, N, C>() * C * (int)sizeof(typename vec2<T>::type);
}
template <typename T, int N, int C> constexpr bool col_valid() {
    return C <= N && threads_per_line<T, N>() * C <= 1024 && col_smem_bytes<T, N, C>() <= kMaxSmem;
}

// Launch with programmatic stream serialisation (see pdl_trigger / pdl_wait).
template <typename... P, typename... A>
cudaError_t launch_pdl(void (*kernel)(P...), dim3 grid, dim3 block, int smem, cudaStream_t s, A&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

template <typename T, int N>
cudaError_t launch_row_pass(const typename vec2<T>::type* src, typename vec2<T>::type* dst,
                            const typename tab_of<T>::type* tw, ScreenCoef<T> sc, double* partials,
                            bool diag, int, int*, unsigned, cudaStream_t s) {
    constexpr int RPB = rows_per_block<T, N>(), THREADS = threads_per_line<T, N>() * RPB;
    constexpr int SMEM = row_smem_bytes<T, N>();
    cudaError_t e;
    if (diag) {
        if ((e = ensure_smem<k_row_pass<T, N, true>>(SMEM)) != cudaSuccess) return e;
        e = launch_pdl(k_row_pass<T, N, true>, dim3(N / RPB), dim3(THREADS), SMEM, s, src, dst, tw, sc, partials);
    } else {
        if ((e = ensure_smem<k_row_pass<T, N, false>>(SMEM)) != cudaSuccess) return e;
        e = launch_pdl(k_row_pass<T, N, false>, dim3(N / RPB), dim3(THREADS), SMEM, s, src, dst, tw, sc, partials);
    }
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <typename T, int N, int C>
cudaError_t launch_col_c(const typename vec2<T>::type* src, typename vec2<T>::type* dst,
                         const typename tab_of<T>::type* tw,
                         const typename tab_of<T>::type* px, const typename tab_of<T>::type* py,
                         typename tab_of<T>::type rot, cudaStream_t s) {
    if constexpr (col_valid<T, N, C>()) {
        constexpr int SMEM = col_smem_bytes<T, N, C>();
        cudaError_t e = ensure_smem<k_col_pass<T, N, C>>(SMEM);
        if (e != cudaSuccess) return e;
        k_col_pass<T, N, C><<<N / C, threads_per_line<T, N>() * C, SMEM, s>>>(src, dst, tw, px, py, rot);
        return cudaGetLastError();
    } else {
        return cudaErrorInvalidConfiguration;
    }
}

// Tensor map of an n x n complex state (state layout, see sidx) as n/2 row
// pairs x n columns x 4 words (4-byte words for complex64, 8-byte for
// complex128: the copies move bits, no conversion), boxes of 4 words x C
// columns x 256 row pairs.  cuTensorMapEncodeTiled is a host-only driver call,
// reached through the runtime's entry-point query so that the library needs no
// link to libcuda.
inline cudaError_t encode_field_map(CUtensorMap* map, const void* base, int n, int word_bytes, int cols) {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }();
    if (!fn) return cudaErrorNotSupported;
    const cuuint64_t dims[3] = {4, (cuuint64_t)n, (cuuint64_t)n / 2};
    const cuuint64_t strides[2] = {(cuuint64_t)4 * word_bytes, (cuuint64_t)4 * word_bytes * n};
    const cuuint32_t box[3] = {4, (cuuint32_t)cols, (cuuint32_t)kTmaBoxRows};
    const cuuint32_t estride[3] = {1, 1, 1};
    const CUresult r = fn(map, word_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_UINT32 : CU_TENSOR_MAP_DATA_TYPE_UINT64, 3,
                          const_cast<void*>(base), dims, strides, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <typename T, int N, int C>
cudaError_t launch_col_tma_c(const typename vec2<T>::type* src, typename vec2<T>::type* dst,
                             const typename tab_of<T>::type* tw,
                             const typename tab_of<T>::type* px, const typename tab_of<T>::type* py,
                             typename tab_of<T>::type rot, int* status, unsigned extra_tx, cudaStream_t s) {
    if constexpr (col_valid<T, N, C>() && col_tma_valid<T, N, C>()) {
        constexpr int SMEM = col_smem_bytes<T, N, C>() + kTmaAlignPad;
        CUtensorMap ml, ms;
        cudaError_t e = encode_field_map(&ml, src, N, (int)sizeof(T), C);
        if (e == cudaSuccess) {
            if (static_cast<const void*>(src) == static_cast<const void*>(dst)) ms = ml;
            else e = encode_field_map(&ms, dst, N, (int)sizeof(T), C);
        }
        if (e == cudaSuccess) e = ensure_smem<k_col_pass_tma<T, N, C>>(SMEM);
        if (e != cudaSuccess) return e;
        e = launch_pdl(k_col_pass_tma<T, N, C>, dim3(N / C), dim3(threads_per_line<T, N>() * C), SMEM, s, ml, ms, tw,
                       px, py, rot, status, extra_tx);
        return e != cudaSuccess ? e : cudaGetLastError();
    } else {
        return cudaErrorInvalidConfiguration;
    }
}

template <typename T, int N>
cudaError_t launch_col_pass(const typename vec2<T>::type* src, typename vec2<T>::type* dst,
                            const typename tab_of<T>::type* tw,
                            const typename tab_of<T>::type* px, const typename tab_of<T>::type* py,
                            typename tab_of<T>::type rot, int cols, int* status, unsigned extra_tx,
                            cudaStream_t s) {
    switch (cols) {
        case 1: return launch_col_c<T, N, 1>(src, dst, tw, px, py, rot, s);
        case 2: return launch_col_c<T, N, 2>(src, dst, tw, px, py, rot, s);
        case 4: return launch_col_c<T, N, 4>(src, dst, tw, px, py, rot, s);
        case 8: return launch_col_c<T, N, 8>(src, dst, tw, px, py, rot, s);
        case 16: return launch_col_c<T, N, 16>(src, dst, tw, px, py, rot, s);
        case kColTma | 1: return launch_col_tma_c<T, N, 1>(src, dst, tw, px, py, rot, status, extra_tx, s);
        case kColTma | 2: return launch_col_tma_c<T, N, 2>(src, dst, tw, px, py, rot, status, extra_tx, s);
        case kColTma | 4: return launch_col_tma_c<T, N, 4>(src, dst, tw, px, py, rot, status, extra_tx, s);
        case kColTma | 8: return launch_col_tma_c<T, N, 8>(src, dst, tw, px, py, rot, status, extra_tx, s);
        case kColTma | 16: return launch_col_tma_c<T, N, 16>(src, dst, tw, px, py, rot, status, extra_tx, s);
        default: return cudaErrorInvalidConfiguration;
    }
}

template <typename T, int N>
cudaError_t launch_row_forward(const typename vec2<T>::type* src, typename vec2<T>::type* dst,
                               const typename tab_of<T>::type* tw, cudaStream_t s) {
    constexpr int RPB = rows_per_block<T, N>(), THREADS = threads_per_line<T, N>() * RPB;
    constexpr int SMEM = row_smem_bytes<T, N>();
    cudaError_t e = ensure_smem<k_row_forward<T, N>>(SMEM);
    if (e != cudaSuccess) return e;
    k_row_forward<T, N><<<N / RPB, THREADS, SMEM, s>>>(src, dst, tw);
    return cudaGetLastError();
}

template <typename T, int N, bool COLS, bool INV>
cudaError_t launch_dft_lines(typename vec2<T>::type* data, const typename tab_of<T>::type* tw, cudaStream_t s) {
    constexpr int LPB = dft_lines_per_block<T, N, COLS>(), THREADS = threads_per_line<T, N>() * LPB;
    constexpr int SMEM = line_stride<T, N, LPB>() * LPB * (int)sizeof(typename vec2<T>::type);
    cudaError_t e = ensure_smem<k_dft_lines<T, N, COLS, INV>>(SMEM);
    if (e != cudaSuccess) return e;
    k_dft_lines<T, N, COLS, INV><<<N / LPB, THREADS, SMEM, s>>>(data, tw);
    return cudaGetLastError();
}

template <typename T, int N, bool INV>
cudaError_t launch_dft2_dir(typename vec2<T>::type* data, const typename tab_of<T>::type* tw, cudaStream_t s) {
    cudaError_t e = launch_dft_lines<T, N, false, INV>(data, tw, s);
    if (e != cudaSuccess) return e;
    return launch_dft_lines<T, N, true, INV>(data, tw, s);
}

template <typename T, int N>
cudaError_t launch_dft2(typename vec2<T>::type* data, const typename tab_of<T>::type* tw, bool inverse,
                        cudaStream_t s) {
    return inverse ? launch_dft2_dir<T, N, true>(data, tw, s) : launch_dft2_dir<T, N, false>(data, tw, s);
}

template <typename T, int N>
cudaError_t launch_readout(const typename vec2<T>::type* state, const typename tab_of<T>::type* tw,
                           typename vec2<T>::type* field_out, T* flu_out, double* partials,
                           typename vec2<T>::type unrot, cudaStream_t s) {
    constexpr int RPB = rows_per_block<T, N>(), THREADS = threads_per_line<T, N>() * RPB;
    constexpr int SMEM = row_smem_bytes<T, N>();
    cudaError_t e = ensure_smem<k_readout<T, N>>(SMEM);
    if (e != cudaSuccess) return e;
    k_readout<T, N><<<N / RPB, THREADS, SMEM, s>>>(state, tw, field_out, flu_out, partials, unrot);
    return cudaGetLastError();
}

template <typename T, int N>
cudaError_t launch_loss_seed(const typename vec2<T>::type* state, typename vec2<T>::type* gam,
                             const double* target, const typename tab_of<T>::type* tw, double seed_scale,
                             double* partials, cudaStream_t s) {
    constexpr int RPB = rows_per_block<T, N>(), THREADS = threads_per_line<T, N>() * RPB;
    constexpr int SMEM = row_smem_bytes<T, N>();
    cudaError_t e = ensure_smem<k_loss_seed<T, N>>(SMEM);
    if (e != cudaSuccess) return e;
    k_loss_seed<T, N><<<N / RPB, THREADS, SMEM, s>>>(state, gam, target, tw, seed_scale, partials);
    return cudaGetLastError();
}

template <typename T, int N>
cudaError_t launch_adj_row(typename vec2<T>::type* gam, const typename vec2<T>::type* tn,
                           const typename tab_of<T>::type* tw, AdjCoef<T> ac, double* acc, cudaStream_t s) {
    constexpr int RPB = rows_per_block<T, N>(), THREADS = threads_per_line<T, N>() * RPB;
    constexpr int SMEM = row_smem_bytes<T, N>();
    cudaError_t e = ensure_smem<k_adj_row<T, N>>(SMEM);
    if (e != cudaSuccess) return e;
    k_adj_row<T, N><<<N / RPB, THREADS, SMEM, s>>>(gam, tn, tw, ac, acc);
    return cudaGetLastError();
}

template <typename T, int N, int C> constexpr bool col_tma_ok() {
    return col_valid<T, N, C>() && col_tma_valid<T, N, C>();
}
template <typename T, int N> constexpr int col_mask() {
    return (col_valid<T, N, 1>() ? 1 : 0) | (col_valid<T, N, 2>() ? 2 : 0) |
           (col_valid<T, N, 4>() ? 4 : 0) | (col_valid<T, N, 8>() ? 8 : 0) |
           (col_valid<T, N, 16>() ? 16 : 0) | (col_tma_ok<T, N, 1>() ? 32 : 0) |
           (col_tma_ok<T, N, 2>() ? 64 : 0) | (col_tma_ok<T, N, 4>() ? 128 : 0) |
           (col_tma_ok<T, N, 8>() ? 256 : 0) | (col_tma_ok<T, N, 16>() ? 512 : 0);
}

// default column tile: the staged single-column tile where it exists (n >=
// 512) -- the fastest or within 2 % of the fastest tile at every size
// measured on GB300 --, else the widest valid tile of at most 512 threads,
// unless its row segments are shorter than one 32-byte sector, in which case
// the narrowest valid tile that fills a sector (else the widest valid tile)
template <typename T, int N> constexpr int col_default() {
    constexpr int cs = 2 * (int)sizeof(T);
    if (col_tma_ok<T, N, 1>()) return kColTma | 1;
    int best = 0;
    for (int i = 0; i < 5; ++i) {
        const int c = kColOptions[i];
        if (((col_mask<T, N>() >> i) & 1) && threads_per_line<T, N>() * c <= 512) best = c;
    }
    if (best * cs >= 32) return best;
    for (int i = 0; i < 5; ++i)
        if (((col_mask<T, N>() >> i) & 1) && kColOptions[i] * cs >= 32) return kColOptions[i];
    for (int i = 0; i < 5; ++i)
        if ((col_mask<T, N>() >> i) & 1) best = kColOptions[i];
    return best;
}

template <typename T, int N> KernelSet<T> make_set() {
    KernelSet<T> k;
    k.n = N;
    k.row_blocks = N / rows_per_block<T, N>();
    k.row_blocks8 = k.row_blocks;
    k.adj_blocks = k.row_blocks;
    k.col_mask = col_mask<T, N>();
    k.col_default = col_default<T, N>();
    k.row_radix_mask = 2;  // the single-line engine of fft.cuh: radix 8 in FP64
    k.row_radix_default = 8;
    k.row_pass = &launch_row_pass<T, N>;
    k.col_pass = &launch_col_pass<T, N>;
    k.row_forward = &launch_row_forward<T, N>;
    k.readout = &launch_readout<T, N>;
    k.loss_seed = &launch_loss_seed<T, N>;
    k.adj_row = &launch_adj_row<T, N>;
    k.dft2 = &launch_dft2<T, N>;
    return k;
}

// defined in nlse_f32.cu / nlse_f64.cu: table for n = 2^log2n, or nullptr
const KernelSet<float>* kernels_f32(int log2n);
const KernelSet<double>* kernels_f64(int log2n);

}  // namespace nlse
