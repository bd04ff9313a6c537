// nlse_f32.cu -- FP32 (complex64) instantiations of the march kernels.
#include "dispatch.cuh"

namespace nlse {

static const KernelSet<float> g_f32[] = {
    make_set<float, 8>(),    make_set<float, 16>(),   make_set<float, 32>(),
    make_set<float, 64>(),   make_set<float, 128>(),  make_set<float, 256>(),
    make_set<float, 512>(),  make_set<float, 1024>(), make_set<float, 2048>(),
    make_set<float, 4096>(), make_set<float, 8192>(),
};

const KernelSet<float>* kernels_f32(int log2n) {
    if (log2n < 3 || log2n > 13) return nullptr;
    return &g_f32[log2n - 3];
}

}  // namespace nlse
