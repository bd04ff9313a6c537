// nlse_f32.cu -- FP32 (complex64) instantiations of the march kernels (the
// pair engine, pass32.cuh).
#include "dispatch32.cuh"

namespace nlse {

static const KernelSet<float> g_f32[] = {
    make_set32<8>(),    make_set32<16>(),   make_set32<32>(),
    make_set32<64>(),   make_set32<128>(),  make_set32<256>(),
    make_set32<512>(),  make_set32<1024>(), make_set32<2048>(),
    make_set32<4096>(), make_set32<8192>(),
};

const KernelSet<float>* kernels_f32(int log2n) {
    if (log2n < 3 || log2n > 13) return nullptr;
    return &g_f32[log2n - 3];
}

}  // namespace nlse
