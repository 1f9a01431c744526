// Power-of-two kernels (rows, f32): explicit instantiations of kernels_p2.cuh.
#include "kernels_p2.cuh"

namespace dgt {
template cudaError_t p2_fft_post<float>(const cplx<float>*, cplx<float>*, const SepGeom&, int64_t, const void*, const PostParams<cplx<float>>&, int64_t, cudaStream_t);
template cudaError_t p2_pre_ifft<float>(const cplx<float>*, cplx<float>*, const SepGeom&, int64_t, const void*, const PostParams<cplx<float>>&, int64_t, cudaStream_t);
template cudaError_t p2_fir_analysis<float>(const void*, int, cplx<float>*, const FirParams<cplx<float>>&, const void*, int64_t, cudaStream_t);
template cudaError_t p2_fir_synthesis<float>(const cplx<float>*, void*, int, cplx<float>*, const FirParams<cplx<float>>&, const void*, int64_t, cudaStream_t);
template int64_t p2_fir_synthesis_cols<float>(int64_t, int64_t, int64_t, int64_t);
}  // namespace dgt
