// Power-of-two kernels (rows, f64): explicit instantiations of kernels_p2.cuh.
#include "kernels_p2.cuh"

namespace dgt {
template cudaError_t p2_fft_post<double>(const cplx<double>*, cplx<double>*, const SepGeom&, int64_t, const void*, const PostParams<cplx<double>>&, int64_t, cudaStream_t);
template cudaError_t p2_pre_ifft<double>(const cplx<double>*, cplx<double>*, const SepGeom&, int64_t, const void*, const PostParams<cplx<double>>&, int64_t, cudaStream_t);
template cudaError_t p2_fir_analysis<double>(const void*, int, cplx<double>*, const FirParams<cplx<double>>&, const void*, int64_t, cudaStream_t);
template cudaError_t p2_fir_synthesis<double>(const cplx<double>*, void*, int, cplx<double>*, const FirParams<cplx<double>>&, const void*, int64_t, cudaStream_t);
template int64_t p2_fir_synthesis_cols<double>(int64_t, int64_t, int64_t, int64_t);
}  // namespace dgt
