// rtt_tc.cu -- tensor-core (tcgen05, BF16 hi/lo split) form of the site chain.
#include "rtt_internal.cuh"

bool tc_supported_chi(int) { return false; }
rtt_status tc_plan_create(rtt_s *, const double *, const double *, const double *) {
    return RTT_ERR_UNSUPPORTED;
}
void tc_plan_destroy(rtt_s *) {}
rtt_status tc_left_env(rtt_s *, const uint8_t *, int64_t, cudaStream_t) { return RTT_ERR_UNSUPPORTED; }
rtt_status tc_right_env(rtt_s *, const uint8_t *, int64_t, cudaStream_t) { return RTT_ERR_UNSUPPORTED; }
rtt_status tc_rows(rtt_s *, const uint8_t *, int64_t, cudaStream_t) { return RTT_ERR_UNSUPPORTED; }
rtt_status tc_chain_init(rtt_s *, const uint8_t *, int64_t, double *, int8_t *, rtt_chain_state *,
                         cudaStream_t) {
    return RTT_ERR_UNSUPPORTED;
}
rtt_status tc_sweep(rtt_s *, uint8_t *, rtt_chain_state *, int64_t, int64_t, int64_t, int32_t,
                    int64_t *, cudaStream_t) {
    return RTT_ERR_UNSUPPORTED;
}
