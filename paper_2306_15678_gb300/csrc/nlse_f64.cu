// nlse_f64.cu -- FP64 (complex128) instantiations of the march kernels.
#include "dispatch.cuh"

namespace nlse {

static const KernelSet<double> g_f64[] = {
    make_set<double, 8>(),    make_set<double, 16>(),   make_set<double, 32>(),
    make_set<double, 64>(),   make_set<double, 128>(),  make_set<double, 256>(),
    make_set<double, 512>(),  make_set<double, 1024>(), make_set<double, 2048>(),
    make_set<double, 4096>(), make_set<double, 8192>(),
};

const KernelSet<double>* kernels_f64(int log2n) {
    if (log2n < 3 || log2n > 13) return nullptr;
    return &g_f64[log2n - 3];
}

}  // namespace nlse
