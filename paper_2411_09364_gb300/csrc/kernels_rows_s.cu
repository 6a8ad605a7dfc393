// Compile-time-size FP32 row transforms: periodic x rows of n = 256, 512 and
// 1536 (complex length L = 128, 256, 768), the sizes of the channel and duct
// workloads.  Other sizes and kinds use the run-time-size kernels.
#include "xy_impl.cuh"

namespace cales {

template <int LS>
static cudaError_t rows_fwd_l(const RowArgs<float>& a, int in_kind, cudaStream_t st) {
    switch (in_kind) {
        case 1: return launch_rows_forward_v<float, double, LS, KIND_P>(a, st);
        case 2: return launch_rows_forward_v<float, RUIn, LS, KIND_P>(a, st);
        default: return launch_rows_forward_v<float, float, LS, KIND_P>(a, st);
    }
}

template <int LS>
static cudaError_t rows_inv_l(const RowArgs<float>& a, int mode, cudaStream_t st) {
    switch (mode) {
        case OUT_T: return launch_rows_inverse_v<float, OUT_T, LS, KIND_P>(a, st);
        case OUT_F64: return launch_rows_inverse_v<float, OUT_F64, LS, KIND_P>(a, st);
        case OUT_FF_INIT: return launch_rows_inverse_v<float, OUT_FF_INIT, LS, KIND_P>(a, st);
        case OUT_FF_ACC: return launch_rows_inverse_v<float, OUT_FF_ACC, LS, KIND_P>(a, st);
        case OUT_FF_ACC_D: return launch_rows_inverse_v<float, OUT_FF_ACC_D, LS, KIND_P>(a, st);
        default: return launch_rows_inverse_v<float, OUT_FF_FINAL, LS, KIND_P>(a, st);
    }
}

bool launch_rows_forward_static(const RowArgs<float>& a, int in_kind, cudaStream_t st, cudaError_t* err) {
    if (!static_fft_enabled() || a.t.kind != KIND_P || !radices_match(a.t, a.t.L)) return false;
    switch (a.t.L) {
        case 128: *err = rows_fwd_l<128>(a, in_kind, st); return true;
        case 256: *err = rows_fwd_l<256>(a, in_kind, st); return true;
        case 768: *err = rows_fwd_l<768>(a, in_kind, st); return true;
        default: return false;
    }
}

bool launch_rows_inverse_static(const RowArgs<float>& a, int mode, cudaStream_t st, cudaError_t* err) {
    if (!static_fft_enabled() || a.t.kind != KIND_P || mode < OUT_T || mode > OUT_FF_ACC_D || !radices_match(a.t, a.t.L))
        return false;
    switch (a.t.L) {
        case 128: *err = rows_inv_l<128>(a, mode, st); return true;
        case 256: *err = rows_inv_l<256>(a, mode, st); return true;
        case 768: *err = rows_inv_l<768>(a, mode, st); return true;
        default: return false;
    }
}

}  // namespace cales
