// Launchers of the x and y transform kernels (templates in xy_impl.cuh): the
// compile-time-size FP32 variants where the sizes have one, else the
// run-time-size kernels instantiated here.
#include "xy_impl.cuh"

#include <cstdlib>
#include <type_traits>

namespace cales {

bool static_fft_enabled() {
    static const bool on = [] {
        const char* e = getenv("CALES_STATIC_FFT");
        return !(e && e[0] == '0');
    }();
    return on;
}

template <typename T, typename TIn>
cudaError_t launch_rows_forward(const RowArgs<T>& a, cudaStream_t st) {
    if constexpr (sizeof(T) == 4) {
        cudaError_t err = cudaSuccess;
        const int in_kind = std::is_same<TIn, RUIn>::value ? 2 : (sizeof(TIn) == 8 ? 1 : 0);
        if (launch_rows_forward_static(a, in_kind, st, &err)) return err;
    }
    return launch_rows_forward_v<T, TIn, 0, -1>(a, st);
}

template <typename T, int MODE>
cudaError_t launch_rows_inverse(const RowArgs<T>& a, cudaStream_t st) {
    if constexpr (sizeof(T) == 4) {
        cudaError_t err = cudaSuccess;
        if (launch_rows_inverse_static(a, MODE, st, &err)) return err;
    }
    return launch_rows_inverse_v<T, MODE, 0, -1>(a, st);
}

template <typename T>
cudaError_t launch_cols(const ColArgs<T>& a, bool inverse, cudaStream_t st) {
    if constexpr (sizeof(T) == 4) {
        cudaError_t err = cudaSuccess;
        if (launch_cols_static(a, inverse, st, &err)) return err;
    }
    switch (a.tx) {
        case 128: return launch_cols_v<T, 128, 0, -1>(a, inverse, st);
        case 64: return launch_cols_v<T, 64, 0, -1>(a, inverse, st);
        case 32: return launch_cols_v<T, 32, 0, -1>(a, inverse, st);
        case 16: return launch_cols_v<T, 16, 0, -1>(a, inverse, st);
        case 8: return launch_cols_v<T, 8, 0, -1>(a, inverse, st);
        default: return launch_cols_v<T, 4, 0, -1>(a, inverse, st);
    }
}

template cudaError_t launch_rows_forward<double, double>(const RowArgs<double>&, cudaStream_t);
template cudaError_t launch_rows_forward<float, float>(const RowArgs<float>&, cudaStream_t);
template cudaError_t launch_rows_forward<float, double>(const RowArgs<float>&, cudaStream_t);
template cudaError_t launch_rows_forward<float, RUIn>(const RowArgs<float>&, cudaStream_t);

bool rows_forward_ru_ok(const RowArgs<float>& a) {
    const auto al16 = [](const void* p) { return ((uintptr_t)p & 15u) == 0; };
    return a.t.n >= 4 && a.t.n % 4 == 0 && al16(a.ru.r) && al16(a.ru.d) && a.ru.nx == a.t.n;
}
template cudaError_t launch_rows_inverse<double, OUT_T>(const RowArgs<double>&, cudaStream_t);
template cudaError_t launch_rows_inverse<float, OUT_T>(const RowArgs<float>&, cudaStream_t);
template cudaError_t launch_rows_inverse<float, OUT_F64>(const RowArgs<float>&, cudaStream_t);
template cudaError_t launch_rows_inverse<float, OUT_FF_INIT>(const RowArgs<float>&, cudaStream_t);
template cudaError_t launch_rows_inverse<float, OUT_FF_ACC>(const RowArgs<float>&, cudaStream_t);
template cudaError_t launch_rows_inverse<float, OUT_FF_FINAL>(const RowArgs<float>&, cudaStream_t);
template cudaError_t launch_rows_inverse<float, OUT_FF_ACC_D>(const RowArgs<float>&, cudaStream_t);
template cudaError_t launch_cols<double>(const ColArgs<double>&, bool, cudaStream_t);
template cudaError_t launch_cols<float>(const ColArgs<float>&, bool, cudaStream_t);

}  // namespace cales
