// Mixed-radix kernels (f64): explicit instantiations of kernels_mr.cuh.
#include "kernels_mr.cuh"

namespace dgt {
template cudaError_t mr_fft_post<double>(const cplx<double>*, cplx<double>*, const SepGeom&, int64_t, const void*, const PostParams<cplx<double>>&, int64_t, cudaStream_t);
template cudaError_t mr_pre_ifft<double>(const cplx<double>*, cplx<double>*, const SepGeom&, int64_t, const void*, const PostParams<cplx<double>>&, int64_t, cudaStream_t);
template cudaError_t mr_zak_fwd<double>(const void*, int, int64_t, cplx<double>*, int64_t, int64_t, int64_t, const void*, const ChirpParams<cplx<double>>&, int64_t, cudaStream_t);
template cudaError_t mr_prod_ifft<double>(const cplx<double>*, const cplx<double>*, int64_t, cplx<double>*, const SepGeom&, const void*, int64_t, cudaStream_t);
template cudaError_t mr_fft_prod_adj<double>(const cplx<double>*, const cplx<double>*, int64_t, cplx<double>*, const SepGeom&, const void*, int64_t, cudaStream_t);
template cudaError_t mr_zak_inv<double>(const cplx<double>*, int64_t, void*, int, int64_t, int64_t, int64_t, const void*, const ChirpParams<cplx<double>>&, double, int64_t, cudaStream_t);
template cudaError_t mr_fftL_cols<double>(const void*, int, cplx<double>*, int64_t, int64_t, int, const void*, const ChirpParams<cplx<double>>&, const CisTable<cplx<double>>&, int64_t, cudaStream_t);
template cudaError_t mr_fftL_rows<double>(const cplx<double>*, void*, int, int64_t, int64_t, int, const void*, const ChirpParams<cplx<double>>&, double, int64_t, cudaStream_t);
}  // namespace dgt
