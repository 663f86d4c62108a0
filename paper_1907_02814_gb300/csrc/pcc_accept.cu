// Diagnostic entry point: the accept decision of the collision kernels
// (Eq. proba3, U < p with the digit-by-digit uniform of accept_u) for given
// 16-bit accept digits and probabilities, in FP64 as the plain path takes it
// and with p rounded to FP32 as the batched path takes it.  It lets the tests
// force the tie a = floor(2^16 p), which the collision kernels reach with
// probability 2^-16 per evaluated pair.
#include <cuda_runtime.h>

#include <algorithm>

#include "pcc_internal.h"

using namespace pcc;

namespace {

__global__ void accept_check_kernel(int n, const uint32_t* __restrict__ r, const double* __restrict__ p,
                                    const uint32_t* __restrict__ c0, const uint32_t* __restrict__ cell,
                                    const uint32_t* __restrict__ tag, uint64_t step, uint64_t seed,
                                    int* __restrict__ out32, int* __restrict__ out64)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const AcceptSrc src{c0[i], cell[i], tag[i]};
        out64[i] = accept_u<double>(r[i], p[i], src, step, seed) ? 1 : 0;
        out32[i] = accept_u<float>(r[i], (float)p[i], src, step, seed) ? 1 : 0;
    }
}

}  // namespace

extern "C" int pcc_accept_check(int n, const uint32_t* r, const double* p, const uint32_t* c0, const uint32_t* cell,
                                const uint32_t* tag, uint64_t step, uint64_t seed, int* out32, int* out64,
                                void* stream)
{
    if (n < 0 || (n > 0 && (!r || !p || !c0 || !cell || !tag || !out32 || !out64))) {
        set_error("pcc_accept_check: invalid argument");
        return PCC_E_INVALID;
    }
    if (n == 0) return PCC_OK;
    const int blocks = (int)std::min<long long>((n + 255) / 256, 4096);
    accept_check_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(n, r, p, c0, cell, tag, step, seed, out32,
                                                                  out64);
    note_launches(1);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PCC_OK : cuda_fail(e, "pcc_accept_check");
}
