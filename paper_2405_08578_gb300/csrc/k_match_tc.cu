// BF16 tensor-core matching (tcgen05) -- under construction.
#include "lp_internal.cuh"

namespace lp {

size_t match_bf16_workspace(int64_t NA, int64_t NB, int num_sms)
{
    (void)NA; (void)NB; (void)num_sms;
    return 256;
}

cudaError_t launch_match_bf16(const MatchArgs& a, void* ws, size_t ws_bytes, int num_sms, cudaStream_t s)
{
    (void)a; (void)ws; (void)ws_bytes; (void)num_sms; (void)s;
    return cudaErrorNotSupported;
}

}  // namespace lp
