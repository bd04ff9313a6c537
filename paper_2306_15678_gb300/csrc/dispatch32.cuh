// dispatch32.cuh -- host-side launchers of the FP32 march kernels of the pair
// engine (pass32.cuh) for every grid size n = 2^k (8..8192), gathered into the
// same per-size tables as the FP64 kernels (dispatch.cuh).  The FP32 kernels
// keep the table's signatures: `tw` is the start of the step's twiddle block
// (pass32.cuh: tw32_*), px holds n entries (x, y), py n/2 pair entries, and
// the state pointers address the unit layout.
#pragma once
#include "dispatch.cuh"
#include "pass32.cuh"

namespace nlse {

template <int N, int E, int C> constexpr bool p_col_valid() {
    return C <= N && p_col_tpl<N, E>() * C <= 1024 && p_col_smem<N, E, C>() <= kMaxSmem;
}
template <int N, int E, int C> constexpr bool p_col_tma_ok() {
    return p_col_valid<N, E, C>() && p_col_tma_valid<N, E, C>();
}

inline const unsigned char* twb_of(const float2* tw) { return reinterpret_cast<const unsigned char*>(tw); }

template <int N, int E>
cudaError_t launch_row_pass32_e(const float2* src, float2* dst, const float2* tw, ScreenCoef<float> sc,
                                double* partials, bool diag, cudaStream_t s) {
    constexpr int THREADS = p_row_threads<N, E>(), SMEM = p_row_smem<N, E>(), BLOCKS = N / 2 / p_rows<N, E>();
    const float4* in = reinterpret_cast<const float4*>(src);
    float4* out = reinterpret_cast<float4*>(dst);
    cudaError_t e;
    constexpr int RES = p_min_blocks<THREADS, E>();  // resident blocks per SM (register limit)
    if (diag) {
        if ((e = ensure_smem_carveout<k_row_pass32<N, E, true>>(SMEM, RES)) != cudaSuccess) return e;
        e = launch_pdl(k_row_pass32<N, E, true>, dim3(BLOCKS), dim3(THREADS), SMEM, s, in, out, twb_of(tw), sc,
                       partials);
    } else {
        if ((e = ensure_smem_carveout<k_row_pass32<N, E, false>>(SMEM, RES)) != cudaSuccess) return e;
        e = launch_pdl(k_row_pass32<N, E, false>, dim3(BLOCKS), dim3(THREADS), SMEM, s, in, out, twb_of(tw), sc,
                       partials);
    }
    return e != cudaSuccess ? e : cudaGetLastError();
}
// the persistent staged row pass exists where a row pair fills whole warps of one block
template <int N> constexpr bool p_row_staged_ok() { return p_rows<N, 16>() == 1 && p_tpl<N, 16>() % 32 == 0; }

// blocks of the persistent row pass: as many as are resident at once
inline int resident_grid(int per_sm, int units) {
    static int sms[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return units;
    if (sms[dev] == 0 && cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return units;
    const long long g = (long long)sms[dev] * per_sm;
    return g < units ? (int)g : units;
}

template <int N>
cudaError_t launch_row_pass32_pf(const float2* src, float2* dst, const float2* tw, ScreenCoef<float> sc,
                                 double* partials, bool diag, int* status, unsigned extra_tx, cudaStream_t s) {
    if constexpr (p_row_staged_ok<N>()) {
        constexpr int THREADS = p_tpl<N, 16>(), SMEM = p_row_smem<N, 16>();
        constexpr int RES = p_min_blocks<THREADS, 16>();
        const float4* in = reinterpret_cast<const float4*>(src);
        float4* out = reinterpret_cast<float4*>(dst);
        const int grid = resident_grid(RES, N / 2);
        cudaError_t e;
        if (diag) {
            if ((e = ensure_smem_carveout<k_row_pass32_pf<N, true>>(SMEM, RES)) != cudaSuccess) return e;
            e = launch_pdl(k_row_pass32_pf<N, true>, dim3(grid), dim3(THREADS), SMEM, s, in, out, twb_of(tw), sc,
                           partials, status, extra_tx);
        } else {
            if ((e = ensure_smem_carveout<k_row_pass32_pf<N, false>>(SMEM, RES)) != cudaSuccess) return e;
            e = launch_pdl(k_row_pass32_pf<N, false>, dim3(grid), dim3(THREADS), SMEM, s, in, out, twb_of(tw), sc,
                           partials, status, extra_tx);
        }
        return e != cudaSuccess ? e : cudaGetLastError();
    } else {
        return cudaErrorInvalidConfiguration;
    }
}

template <int N>
cudaError_t launch_row_pass32(const float2* src, float2* dst, const float2* tw, ScreenCoef<float> sc,
                              double* partials, bool diag, int rad, int* status, unsigned extra_tx, cudaStream_t s) {
    if (rad == 16) return launch_row_pass32_e<N, 16>(src, dst, tw, sc, partials, diag, s);
    if (rad == 8) return launch_row_pass32_e<N, 8>(src, dst, tw, sc, partials, diag, s);
    if (rad == (kRowStaged | 16))
        return launch_row_pass32_pf<N>(src, dst, tw, sc, partials, diag, status, extra_tx, s);
    return cudaErrorInvalidConfiguration;
}

template <int N, int E, int C>
cudaError_t launch_col32_c(const float2* src, float2* dst, const float2* tw, const float2* px, const float2* py,
                           float2 rot, cudaStream_t s) {
    if constexpr (p_col_valid<N, E, C>()) {
        constexpr int SMEM = p_col_smem<N, E, C>();
        cudaError_t e = ensure_smem_carveout<k_col_pass32<N, E, C>>(SMEM, p_col_min_blocks<p_col_tpl<N, E>() * C, E>());
        if (e != cudaSuccess) return e;
        e = launch_pdl(k_col_pass32<N, E, C>, dim3(N / C), dim3(p_col_tpl<N, E>() * C), SMEM, s,
                       reinterpret_cast<const float4*>(src), reinterpret_cast<float4*>(dst), twb_of(tw), px,
                       reinterpret_cast<const float4*>(py), rot);
        return e != cudaSuccess ? e : cudaGetLastError();
    } else {
        return cudaErrorInvalidConfiguration;
    }
}

template <int N, int E, int C>
cudaError_t launch_col32_tma_c(const float2* src, float2* dst, const float2* tw, const float2* px,
                               const float2* py, float2 rot, int* status, unsigned extra_tx, cudaStream_t s) {
    if constexpr (p_col_tma_ok<N, E, C>()) {
        constexpr int SMEM = p_col_smem<N, E, C>() + kTmaAlignPad;
        CUtensorMap ml, ms;
        // boxes of one column: every column of the tile lands at its own line
        cudaError_t e = encode_field_map(&ml, src, N, 4, 1);
        if (e == cudaSuccess) {
            if (static_cast<const void*>(src) == static_cast<const void*>(dst)) ms = ml;
            else e = encode_field_map(&ms, dst, N, 4, 1);
        }
        if (e == cudaSuccess)
            e = ensure_smem_carveout<k_col_pass32_tma<N, E, C>>(SMEM, p_col_min_blocks<p_col_tpl<N, E>() * C, E>());
        if (e != cudaSuccess) return e;
        e = launch_pdl(k_col_pass32_tma<N, E, C>, dim3(N / C), dim3(p_col_tpl<N, E>() * C), SMEM, s, ml, ms,
                       twb_of(tw), px, reinterpret_cast<const float4*>(py), rot, status, extra_tx);
        return e != cudaSuccess ? e : cudaGetLastError();
    } else {
        return cudaErrorInvalidConfiguration;
    }
}

template <int N, int E>
cudaError_t launch_col_pass32_e(const float2* src, float2* dst, const float2* tw, const float2* px,
                                const float2* py, float2 rot, int cols, int* status, unsigned extra_tx,
                                cudaStream_t s) {
    switch (cols & ~kColR8) {
        case 1: return launch_col32_c<N, E, 1>(src, dst, tw, px, py, rot, s);
        case 2: return launch_col32_c<N, E, 2>(src, dst, tw, px, py, rot, s);
        case 4: return launch_col32_c<N, E, 4>(src, dst, tw, px, py, rot, s);
        case 8: return launch_col32_c<N, E, 8>(src, dst, tw, px, py, rot, s);
        case 16: return launch_col32_c<N, E, 16>(src, dst, tw, px, py, rot, s);
        case kColTma | 1: return launch_col32_tma_c<N, E, 1>(src, dst, tw, px, py, rot, status, extra_tx, s);
        case kColTma | 2: return launch_col32_tma_c<N, E, 2>(src, dst, tw, px, py, rot, status, extra_tx, s);
        case kColTma | 4: return launch_col32_tma_c<N, E, 4>(src, dst, tw, px, py, rot, status, extra_tx, s);
        case kColTma | 8: return launch_col32_tma_c<N, E, 8>(src, dst, tw, px, py, rot, status, extra_tx, s);
        case kColTma | 16: return launch_col32_tma_c<N, E, 16>(src, dst, tw, px, py, rot, status, extra_tx, s);
        default: return cudaErrorInvalidConfiguration;
    }
}
template <int N>
cudaError_t launch_col_pass32(const float2* src, float2* dst, const float2* tw, const float2* px, const float2* py,
                              float2 rot, int cols, int* status, unsigned extra_tx, cudaStream_t s) {
    if (cols & kColR8) return launch_col_pass32_e<N, 8>(src, dst, tw, px, py, rot, cols, status, extra_tx, s);
    return launch_col_pass32_e<N, 16>(src, dst, tw, px, py, rot, cols, status, extra_tx, s);
}

template <int N> cudaError_t launch_row_forward32(const float2* src, float2* dst, const float2* tw, cudaStream_t s) {
    constexpr int THREADS = p_row_threads<N, 16>(), SMEM = p_row_smem<N, 16>(), BLOCKS = N / 2 / p_rows<N, 16>();
    cudaError_t e = ensure_smem<k_row_forward32<N>>(SMEM);
    if (e != cudaSuccess) return e;
    k_row_forward32<N><<<BLOCKS, THREADS, SMEM, s>>>(src, reinterpret_cast<float4*>(dst), twb_of(tw));
    return cudaGetLastError();
}

template <int N>
cudaError_t launch_readout32(const float2* state, const float2* tw, float2* field_out, float* flu_out,
                             double* partials, float2 unrot, cudaStream_t s) {
    constexpr int THREADS = p_row_threads<N, 16>(), SMEM = p_row_smem<N, 16>(), BLOCKS = N / 2 / p_rows<N, 16>();
    cudaError_t e = ensure_smem<k_readout32<N>>(SMEM);
    if (e != cudaSuccess) return e;
    k_readout32<N><<<BLOCKS, THREADS, SMEM, s>>>(reinterpret_cast<const float4*>(state), twb_of(tw), field_out,
                                                 flu_out, partials, unrot);
    return cudaGetLastError();
}

template <int N>
cudaError_t launch_loss_seed32(const float2* state, float2* gam, const double* target, const float2* tw,
                               double seed_scale, double* partials, cudaStream_t s) {
    constexpr int RPB = rows_per_block<float, N>(), THREADS = threads_per_line<float, N>() * RPB;
    constexpr int SMEM = row_smem_bytes<float, N>();
    cudaError_t e = ensure_smem<k_loss_seed32<N>>(SMEM);
    if (e != cudaSuccess) return e;
    k_loss_seed32<N><<<N / RPB, THREADS, SMEM, s>>>(reinterpret_cast<const float4*>(state),
                                                    reinterpret_cast<float4*>(gam), target, tw, seed_scale, partials);
    return cudaGetLastError();
}

template <int N>
cudaError_t launch_adj_row32(float2* gam, const float2* tn, const float2* tw, AdjCoef<float> ac, double* acc,
                             cudaStream_t s) {
    constexpr int RPB = rows_per_block<float, N>(), THREADS = threads_per_line<float, N>() * RPB;
    constexpr int SMEM = row_smem_bytes<float, N>();
    cudaError_t e = ensure_smem<k_adj_row32<N>>(SMEM);
    if (e != cudaSuccess) return e;
    k_adj_row32<N><<<N / RPB, THREADS, SMEM, s>>>(reinterpret_cast<float4*>(gam), reinterpret_cast<const float4*>(tn),
                                                  tw, ac, acc);
    return cudaGetLastError();
}

template <int N, int E> constexpr int col_mask32_e() {
    return (p_col_valid<N, E, 1>() ? 1 : 0) | (p_col_valid<N, E, 2>() ? 2 : 0) | (p_col_valid<N, E, 4>() ? 4 : 0) |
           (p_col_valid<N, E, 8>() ? 8 : 0) | (p_col_valid<N, E, 16>() ? 16 : 0) |
           (p_col_tma_ok<N, E, 1>() ? 32 : 0) | (p_col_tma_ok<N, E, 2>() ? 64 : 0) |
           (p_col_tma_ok<N, E, 4>() ? 128 : 0) | (p_col_tma_ok<N, E, 8>() ? 256 : 0) |
           (p_col_tma_ok<N, E, 16>() ? 512 : 0);
}
// bits 0-9: radix-16 tiles, bits 10-19: radix-8 tiles (kColOptions order)
template <int N> constexpr int col_mask32() { return col_mask32_e<N, 16>() | (col_mask32_e<N, 8>() << 10); }

// default column tile (radix 16): the narrowest staged tile of at least 128
// threads (else the widest staged tile), else the narrowest per-thread tile
// of at least 128 threads (else the widest valid tile)
template <int N> constexpr int col_default32() {
    constexpr int m = col_mask32<N>();
    int best = 0;
    for (int i = 5; i < 10; ++i)
        if ((m >> i) & 1) {
            best = kColOptions[i];
            if (p_col_tpl<N, 16>() * (kColOptions[i] & 0xff) >= 128) return best;
        }
    if (best) return best;
    for (int i = 0; i < 5; ++i)
        if ((m >> i) & 1) {
            best = kColOptions[i];
            if (p_col_tpl<N, 16>() * kColOptions[i] >= 128) return best;
        }
    if (best) return best;
    return 1;
}

template <int N> KernelSet<float> make_set32() {
    KernelSet<float> k;
    k.n = N;
    k.row_blocks = N / 2 / p_rows<N, 16>();  // partials of the readout and the radix-16 row pass
    k.row_blocks8 = N / 2 / p_rows<N, 8>();
    k.adj_blocks = N / rows_per_block<float, N>();
    k.col_mask = col_mask32<N>();
    k.col_default = col_default32<N>();
    k.row_radix_mask = 3 | (p_row_staged_ok<N>() ? 4 : 0);
    k.row_radix_default = 16;
    k.row_pass = &launch_row_pass32<N>;
    k.col_pass = &launch_col_pass32<N>;
    k.row_forward = &launch_row_forward32<N>;
    k.readout = &launch_readout32<N>;
    k.loss_seed = &launch_loss_seed32<N>;
    k.adj_row = &launch_adj_row32<N>;
    k.dft2 = &launch_dft2<float, N>;
    return k;
}

}  // namespace nlse
