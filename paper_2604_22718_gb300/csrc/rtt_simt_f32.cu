// rtt_simt_f32.cu -- FP32 instantiation of the SIMT kernels (rtt_simt.cuh).
#include "rtt_simt.cuh"

RTT_DEFINE_SIMT(float, f32)
