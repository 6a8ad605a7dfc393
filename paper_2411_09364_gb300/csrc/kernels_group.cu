// Launchers of the grouped transform and z kernels (one launch per stage of a
// batch of solves; kernel templates in xy_impl.cuh and z_impl.cuh).
#include "xy_impl.cuh"
#include "z_impl.cuh"

namespace cales {

template <typename T> size_t rows_smem_bytes(const RowArgs<T>& a) {
    return RowLayout<T>(a.rpc, a.t.L > 0 ? a.t.L : 1, a.t.n, a.t.kind, a.t.twlen, 0).total;
}

template <typename T> size_t cols_smem_bytes(const ColArgs<T>& a) {
    return col_smem<T>(a.tx, a.t.L, a.t.kind, a.t.twlen);
}

template <typename K> static cudaError_t set_smem(K kern, size_t smem) {
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <typename T, typename TIn>
cudaError_t launch_rows_forward_grp(const RowArgs<T>* items, const int2* work, int nblocks, size_t smem,
                                    cudaStream_t st) {
    auto kern = k_rows_forward_grp<T, TIn>;
    set_smem(kern, smem);
    kern<<<(unsigned)nblocks, 256, smem, st>>>(items, work);
    return cudaGetLastError();
}

template <typename T, int MODE>
cudaError_t launch_rows_inverse_grp(const RowArgs<T>* items, const int2* work, int nblocks, size_t smem,
                                    cudaStream_t st) {
    auto kern = k_rows_inverse_grp<T, MODE>;
    set_smem(kern, smem);
    kern<<<(unsigned)nblocks, 256, smem, st>>>(items, work);
    return cudaGetLastError();
}

template <typename T, int TX>
static cudaError_t cols_grp_tx(const ColArgs<T>* items, const int2* work, int nblocks, bool inverse, size_t smem,
                               cudaStream_t st) {
    auto kern = inverse ? k_cols_grp<T, TX, true> : k_cols_grp<T, TX, false>;
    set_smem(kern, smem);
    kern<<<(unsigned)nblocks, 256, smem, st>>>(items, work);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cols_grp(const ColArgs<T>* items, const int2* work, int nblocks, int tx, bool inverse, size_t smem,
                            cudaStream_t st) {
    switch (tx) {
        case 128: return cols_grp_tx<T, 128>(items, work, nblocks, inverse, smem, st);
        case 64: return cols_grp_tx<T, 64>(items, work, nblocks, inverse, smem, st);
        case 32: return cols_grp_tx<T, 32>(items, work, nblocks, inverse, smem, st);
        case 16: return cols_grp_tx<T, 16>(items, work, nblocks, inverse, smem, st);
        case 8: return cols_grp_tx<T, 8>(items, work, nblocks, inverse, smem, st);
        case 4: return cols_grp_tx<T, 4>(items, work, nblocks, inverse, smem, st);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T, int MAXM>
static cudaError_t z_grp_m(const ZArgs<T>* items, const int2* work, int nblocks, bool adjoint, int threads,
                           size_t smem, cudaStream_t st) {
    auto kern = adjoint ? k_zsolve_w_grp<T, MAXM, true> : k_zsolve_w_grp<T, MAXM, false>;
    set_smem(kern, smem);
    kern<<<(unsigned)nblocks, threads, smem, st>>>(items, work);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_zsolve_grp(const ZArgs<T>* items, const int2* work, int nblocks, int maxm, bool adjoint,
                              int threads, size_t smem, cudaStream_t st) {
    switch (maxm) {
        case 16: return z_grp_m<T, 16>(items, work, nblocks, adjoint, threads, smem, st);
        case 32: return z_grp_m<T, 32>(items, work, nblocks, adjoint, threads, smem, st);
        case 64: return z_grp_m<T, 64>(items, work, nblocks, adjoint, threads, smem, st);
        default: return cudaErrorInvalidValue;
    }
}

template size_t rows_smem_bytes<float>(const RowArgs<float>&);
template size_t rows_smem_bytes<double>(const RowArgs<double>&);
template size_t cols_smem_bytes<float>(const ColArgs<float>&);
template size_t cols_smem_bytes<double>(const ColArgs<double>&);
template size_t zsolve_w_smem_pb<float>(int, int, int);
template size_t zsolve_w_smem_pb<double>(int, int, int);
template cudaError_t launch_rows_forward_grp<float, double>(const RowArgs<float>*, const int2*, int, size_t,
                                                            cudaStream_t);
template cudaError_t launch_rows_forward_grp<float, float>(const RowArgs<float>*, const int2*, int, size_t,
                                                           cudaStream_t);
template cudaError_t launch_rows_inverse_grp<float, OUT_F64>(const RowArgs<float>*, const int2*, int, size_t,
                                                             cudaStream_t);
template cudaError_t launch_rows_inverse_grp<float, OUT_FF_INIT>(const RowArgs<float>*, const int2*, int, size_t,
                                                                 cudaStream_t);
template cudaError_t launch_rows_inverse_grp<float, OUT_FF_ACC>(const RowArgs<float>*, const int2*, int, size_t,
                                                                cudaStream_t);
template cudaError_t launch_rows_inverse_grp<float, OUT_FF_FINAL>(const RowArgs<float>*, const int2*, int, size_t,
                                                                  cudaStream_t);
template cudaError_t launch_cols_grp<float>(const ColArgs<float>*, const int2*, int, int, bool, size_t, cudaStream_t);
template cudaError_t launch_zsolve_grp<float>(const ZArgs<float>*, const int2*, int, int, bool, int, size_t,
                                              cudaStream_t);

}  // namespace cales
