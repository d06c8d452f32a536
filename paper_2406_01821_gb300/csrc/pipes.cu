// Measured issue rates of the arithmetic pipes the kernels use, for their rooflines: the lane
// operations per second of a stream of one instruction kind (FP32 fused multiply-add, FP32
// multiply, the three-input logic op, population count, the special-function unit's base-2
// exponential, and a float compare writing a register), each thread running eight independent
// chains over a grid of 2048 threads per SM so that latency is hidden and only the pipe's rate is
// left. The compiler cannot fold the chains: every operation is inline PTX on a value the
// previous one produced.
#include "rs_internal.cuh"

namespace rs {

namespace {

enum { OP_FFMA, OP_FMUL, OP_LOP3, OP_POPC, OP_EX2, OP_FSET, OP_COUNT };

template <int OP>
__global__ void __launch_bounds__(512) k_pipe(float *sink, int iters, float a, float b, float skey, uint32_t tkey)
{
    float x[8];
    uint32_t u[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        x[i] = a + 0.001f * (float)i + (float)threadIdx.x * 1e-6f;
        u[i] = threadIdx.x * 7u + (uint32_t)i;
    }
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (OP == OP_FFMA) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(x[i]) : "f"(a), "f"(b));
            if (OP == OP_FMUL) asm volatile("mul.rn.f32 %0, %0, %1;" : "+f"(x[i]) : "f"(a));
            if (OP == OP_LOP3) asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(u[i]) : "r"(5u), "r"(3u));
            if (OP == OP_POPC) asm volatile("popc.b32 %0, %0;" : "+r"(u[i]));
            if (OP == OP_EX2) asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+f"(x[i]));
            if (OP == OP_FSET) asm volatile("set.gt.u32.f32 %0, %1, %2;" : "=r"(u[i]) : "f"(__uint_as_float(u[i])), "f"(b));
        }
    }
    float s = 0.f;
    uint32_t t = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        s += x[i];
        t ^= u[i];
    }
    // keys that no chain reaches, known only at run time: every chain stays live
    if (s == skey || t == tkey) sink[blockIdx.x] = s + (float)t;
}

template <int OP>
rs_status time_op(int sms, float *sink, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, double *out)
{
    constexpr int threads = 512, iters = 4096;
    const int blocks = sms * 4;
    k_pipe<OP><<<blocks, threads, 0, st>>>(sink, 16, 1.0001f, 0.5f, -1.5e30f, 0xFFFFFFFFu);   // warm-up
    RS_CUDA(cudaEventRecord(e0, st));
    k_pipe<OP><<<blocks, threads, 0, st>>>(sink, iters, 1.0001f, 0.5f, -1.5e30f, 0xFFFFFFFFu);
    RS_CUDA(cudaEventRecord(e1, st));
    RS_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    RS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    *out = (double)blocks * threads * iters * 8 / (ms * 1e-3);
    return RS_OK;
}

}  // namespace

rs_status measure_pipe_rates(Ctx *ctx, rs_pipe_rates *out)
{
    float *sink = nullptr;
    RS_CUDA(cudaMalloc(&sink, sizeof(float) * 4 * (size_t)ctx->sm_count));
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    rs_status rc = RS_OK;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        rc = cuda_fail(cudaGetLastError(), "pipe rates set-up");
    const int sms = ctx->sm_count;
    if (!rc) rc = time_op<OP_FFMA>(sms, sink, st, e0, e1, &out->ffma);
    if (!rc) rc = time_op<OP_FMUL>(sms, sink, st, e0, e1, &out->fmul);
    if (!rc) rc = time_op<OP_LOP3>(sms, sink, st, e0, e1, &out->lop3);
    if (!rc) rc = time_op<OP_POPC>(sms, sink, st, e0, e1, &out->popc);
    if (!rc) rc = time_op<OP_EX2>(sms, sink, st, e0, e1, &out->ex2);
    if (!rc) rc = time_op<OP_FSET>(sms, sink, st, e0, e1, &out->fset);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    cudaFree(sink);
    return rc;
}

}  // namespace rs
