// Integer-ALU throughput probe for the 16-byte SAD used by the matchers.
// A measurement utility (the paper has no counterpart): every thread keeps a
// reference descriptor and eight candidate descriptors in registers and
// accumulates SAD16 over them in a loop, so the kernel executes nothing but
// the SAD sequence plus one add per eight SADs.  The rate it reaches over all
// SMs is the ALU ceiling the roofline of the SAD kernels is quoted against.
#include "launch.cuh"

namespace elas {

// variant 0: __vabsdiffu4 + __dp4a (the support matcher's sequence)
// variant 1: __vsadu4
// variant 2: PTX vabsdiff4 with accumulate (the dense matcher's sequence)
__device__ __forceinline__ uint32_t sad16_v(const uint4 &a, const uint4 &b, uint32_t acc, int variant) {
    if (variant == 1) {
        return acc + __vsadu4(a.x, b.x) + __vsadu4(a.y, b.y) + __vsadu4(a.z, b.z) + __vsadu4(a.w, b.w);
    } else if (variant == 2) {
        uint32_t r = acc;
        asm("vabsdiff4.u32.u32.u32.add %0, %1, %2, %0;" : "+r"(r) : "r"(a.x), "r"(b.x));
        asm("vabsdiff4.u32.u32.u32.add %0, %1, %2, %0;" : "+r"(r) : "r"(a.y), "r"(b.y));
        asm("vabsdiff4.u32.u32.u32.add %0, %1, %2, %0;" : "+r"(r) : "r"(a.z), "r"(b.z));
        asm("vabsdiff4.u32.u32.u32.add %0, %1, %2, %0;" : "+r"(r) : "r"(a.w), "r"(b.w));
        return r;
    }
    uint32_t s = __dp4a(__vabsdiffu4(a.x, b.x), 0x01010101u, acc);
    s = __dp4a(__vabsdiffu4(a.y, b.y), 0x01010101u, s);
    s = __dp4a(__vabsdiffu4(a.z, b.z), 0x01010101u, s);
    return __dp4a(__vabsdiffu4(a.w, b.w), 0x01010101u, s);
}

template <int VARIANT>
__global__ void sad_probe_kernel(int iters, uint32_t seed, uint32_t *out) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    uint4 b[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const uint32_t z = (t + 1u) * 2654435761u ^ (seed + 97u * k);
        b[k] = make_uint4(z, z * 747796405u, z ^ 0x9E3779B9u, z + 12345u);
    }
    uint4 a = make_uint4(seed ^ t, seed * 3u, t * 7u, seed + t);
    uint32_t acc0 = 0, acc1 = 0;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; k += 2) {
            acc0 = sad16_v(a, b[k], acc0, VARIANT);
            acc1 = sad16_v(a, b[k + 1], acc1, VARIANT);
        }
        // rotate the reference words and fold in a result: every word of `a`
        // meets a different candidate word each iteration, so no partial SAD
        // can be hoisted out of the loop (one add per eight SAD16)
        a = make_uint4(a.y, a.z, a.w, a.x + acc0);
    }
    if ((acc0 ^ acc1) == 0xFFFFFFFFu) out[t] = acc0;  // practically never taken
}

}  // namespace elas

extern "C" elas_status elas_probe_sad16(int32_t variant, int32_t blocks, int32_t threads, int32_t iters,
                                        uint32_t *scratch, elas_stream stream) {
    using namespace elas;
    if (variant < 0 || variant > 2 || blocks < 1 || threads < 32 || threads > 1024 || iters < 1 || !scratch)
        return fail(ELAS_ERR_INVALID_ARG, "bad probe arguments");
    cudaStream_t st = to_stream(stream);
    if (variant == 0) sad_probe_kernel<0><<<blocks, threads, 0, st>>>(iters, 0x1234u, scratch);
    if (variant == 1) sad_probe_kernel<1><<<blocks, threads, 0, st>>>(iters, 0x1234u, scratch);
    if (variant == 2) sad_probe_kernel<2><<<blocks, threads, 0, st>>>(iters, 0x1234u, scratch);
    return launch_status("sad_probe_kernel");
}
