// Power-of-two kernels (cols, f64): explicit instantiations of kernels_p2.cuh.
#include "kernels_p2.cuh"

namespace dgt {
template cudaError_t p2_zak_fwd<double>(const void*, int, int64_t, cplx<double>*, int64_t, int64_t, int64_t, const void*, const ChirpParams<cplx<double>>&, int64_t, cudaStream_t);
template cudaError_t p2_prod_ifft<double>(const cplx<double>*, const cplx<double>*, int64_t, cplx<double>*, const SepGeom&, const void*, int64_t, cudaStream_t);
template cudaError_t p2_fft_prod_adj<double>(const cplx<double>*, const cplx<double>*, int64_t, cplx<double>*, const SepGeom&, const void*, int64_t, unsigned int*, cudaStream_t);
template cudaError_t p2_zak_inv<double>(const cplx<double>*, int64_t, void*, int, int64_t, int64_t, int64_t, const void*, const ChirpParams<cplx<double>>&, double, int64_t, cudaStream_t);
template cudaError_t p2_zak_prod_ifft<double>(const void*, int, int64_t, const cplx<double>*, int64_t, cplx<double>*, const SepGeom&, const void*, const ChirpParams<cplx<double>>&, int64_t, cudaStream_t);
}  // namespace dgt
