// Expected-emission operator (forward and adjoint): see pcc.h.
#include "pcc_internal.h"

using namespace pcc;

extern "C" int pcc_expected_emission_fwd(pcc_ctx* ctx, int, int, int, int, const float*, const float*,
                                         const float*, float*, void*)
{
    (void)ctx;
    set_error("pcc_expected_emission_fwd: not built yet");
    return PCC_E_INVALID;
}

extern "C" int pcc_expected_emission_bwd(pcc_ctx* ctx, int, int, int, int, const float*, const float*,
                                         const float*, const float*, float*, void*)
{
    (void)ctx;
    set_error("pcc_expected_emission_bwd: not built yet");
    return PCC_E_INVALID;
}
