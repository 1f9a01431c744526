// Power-of-two kernels (cols, f32): explicit instantiations of kernels_p2.cuh.
#include "kernels_p2.cuh"

namespace dgt {
template cudaError_t p2_zak_fwd<float>(const void*, int, int64_t, cplx<float>*, int64_t, int64_t, int64_t, const void*, const ChirpParams<cplx<float>>&, int64_t, cudaStream_t);
template cudaError_t p2_prod_ifft<float>(const cplx<float>*, const cplx<float>*, int64_t, cplx<float>*, const SepGeom&, const void*, int64_t, cudaStream_t);
template cudaError_t p2_fft_prod_adj<float>(const cplx<float>*, const cplx<float>*, int64_t, cplx<float>*, const SepGeom&, const void*, int64_t, unsigned int*, cudaStream_t);
template cudaError_t p2_zak_inv<float>(const cplx<float>*, int64_t, void*, int, int64_t, int64_t, int64_t, const void*, const ChirpParams<cplx<float>>&, float, int64_t, cudaStream_t);
template cudaError_t p2_zak_prod_ifft<float>(const void*, int, int64_t, const cplx<float>*, int64_t, cplx<float>*, const SepGeom&, const void*, const ChirpParams<cplx<float>>&, int64_t, cudaStream_t);
}  // namespace dgt
