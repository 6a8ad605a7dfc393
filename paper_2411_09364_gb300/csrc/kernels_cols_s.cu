// Compile-time-size FP32 column transforms: y lengths n = 128, 256, 512
// (complex length L = 64, 128, 256) with the tile widths the plan picks for
// them, for every kind.  Other sizes and tiles use the run-time-size kernels.
#include "xy_impl.cuh"

namespace cales {

template <int LS, int TX>
static cudaError_t cols_l(const ColArgs<float>& a, bool inverse, cudaStream_t st) {
    switch (a.t.kind) {
        case KIND_P: return launch_cols_v<float, TX, LS, KIND_P>(a, inverse, st);
        case KIND_N: return launch_cols_v<float, TX, LS, KIND_N>(a, inverse, st);
        default: return launch_cols_v<float, TX, LS, KIND_D>(a, inverse, st);
    }
}

bool launch_cols_static(const ColArgs<float>& a, bool inverse, cudaStream_t st, cudaError_t* err) {
    if (!static_fft_enabled() || a.t.kind > KIND_D || !radices_match(a.t, a.t.L)) return false;
    if (a.t.L == 64 && a.tx == 32) { *err = cols_l<64, 32>(a, inverse, st); return true; }
    if (a.t.L == 128 && a.tx == 32) { *err = cols_l<128, 32>(a, inverse, st); return true; }
    if (a.t.L == 256 && a.tx == 16) {
        // one-buffer variant (global-memory packing and unpacking)
        switch (a.t.kind) {
            case KIND_P: *err = launch_cols_g<256, KIND_P>(a, inverse, st); break;
            case KIND_N: *err = launch_cols_g<256, KIND_N>(a, inverse, st); break;
            default: *err = launch_cols_g<256, KIND_D>(a, inverse, st); break;
        }
        return true;
    }
    return false;
}

}  // namespace cales
