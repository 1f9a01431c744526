// Mixed-radix kernels (f32): explicit instantiations of kernels_mr.cuh.
#include "kernels_mr.cuh"

namespace dgt {
template cudaError_t mr_fft_post<float>(const cplx<float>*, cplx<float>*, const SepGeom&, int64_t, const void*, const PostParams<cplx<float>>&, int64_t, cudaStream_t);
template cudaError_t mr_pre_ifft<float>(const cplx<float>*, cplx<float>*, const SepGeom&, int64_t, const void*, const PostParams<cplx<float>>&, int64_t, cudaStream_t);
template cudaError_t mr_zak_fwd<float>(const void*, int, int64_t, cplx<float>*, int64_t, int64_t, int64_t, const void*, const ChirpParams<cplx<float>>&, int64_t, cudaStream_t);
template cudaError_t mr_prod_ifft<float>(const cplx<float>*, const cplx<float>*, int64_t, cplx<float>*, const SepGeom&, const void*, int64_t, cudaStream_t);
template cudaError_t mr_fft_prod_adj<float>(const cplx<float>*, const cplx<float>*, int64_t, cplx<float>*, const SepGeom&, const void*, int64_t, cudaStream_t);
template cudaError_t mr_zak_inv<float>(const cplx<float>*, int64_t, void*, int, int64_t, int64_t, int64_t, const void*, const ChirpParams<cplx<float>>&, float, int64_t, cudaStream_t);
template cudaError_t mr_fftL_cols<float>(const void*, int, cplx<float>*, int64_t, int64_t, int, const void*, const ChirpParams<cplx<float>>&, const CisTable<cplx<float>>&, int64_t, cudaStream_t);
template cudaError_t mr_fftL_rows<float>(const cplx<float>*, void*, int, int64_t, int64_t, int, const void*, const ChirpParams<cplx<float>>&, float, int64_t, cudaStream_t);
}  // namespace dgt
