// ts_prop_n128.cu -- propagation pass kernels for N = 128 (separate unit so the N variants compile in parallel).
#include "ts_prop_impl.cuh"

namespace ts {
template cudaError_t row_pass_n<128>(int, int, int, const RowParams&, int, cudaStream_t);
template cudaError_t col_pass_n<128>(int, int, bool, bool, const ColParams&, int, cudaStream_t, bool);
template cudaError_t prepare_prop_n<128>();
}  // namespace ts
