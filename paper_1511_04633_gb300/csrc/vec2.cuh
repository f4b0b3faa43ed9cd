// vec2.cuh -- the number types of the collision: one cell per thread (plain
// float) or two cells per thread (F2, Blackwell's packed f32x2 instructions,
// PTX ISA 8.6, sm_100 and later: one instruction adds, multiplies or fuses a
// multiply-add for both cells).
//
// F2 rounds every operation on its own: PTX with an explicit rounding mode.
// The collision (step_body.cuh) is written so that no product is added or
// subtracted as a separate operation (each such pair is an explicit fma()),
// which leaves the compiler nothing to fuse on either form: a kernel that
// collides two cells per thread with F2 computes bitwise the values that a
// kernel colliding one cell per thread in float computes, lane by lane.
#pragma once

#include <cuda_runtime.h>

namespace lbm {

// One cell: float with the fused multiply-add and reciprocal the collision
// calls.
__device__ __forceinline__ float fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float recip(float a) { return 1.0f / a; }

// Two cells: lane x is the first cell, lane y the second.
struct F2 {
    float2 v;
    F2() = default;
    __device__ __forceinline__ F2(float s) : v(make_float2(s, s)) {}
    __device__ __forceinline__ F2(float a, float b) : v(make_float2(a, b)) {}
    __device__ __forceinline__ explicit F2(float2 p) : v(p) {}
};

// The packed operations are written as PTX with an explicit rounding mode.
// ptxas still fuses a packed multiply into a following packed add or subtract
// (measured on GB300), which is why the collision never writes that pair.
#define DMRT_F2_BINARY(OP, NAME)                                                          \
    __device__ __forceinline__ F2 OP(F2 a, F2 b)                                          \
    {                                                                                     \
        F2 r;                                                                             \
        asm("{\n\t.reg .b64 A, B, D;\n\tmov.b64 A, {%2, %3};\n\tmov.b64 B, {%4, %5};\n\t" \
            NAME " D, A, B;\n\tmov.b64 {%0, %1}, D;\n\t}"                               \
            : "=f"(r.v.x), "=f"(r.v.y)                                                    \
            : "f"(a.v.x), "f"(a.v.y), "f"(b.v.x), "f"(b.v.y));                            \
        return r;                                                                         \
    }
DMRT_F2_BINARY(operator+, "add.rn.f32x2")
DMRT_F2_BINARY(operator-, "sub.rn.f32x2")
DMRT_F2_BINARY(operator*, "mul.rn.f32x2")
#undef DMRT_F2_BINARY

__device__ __forceinline__ F2 fma(F2 a, F2 b, F2 c)
{
    F2 r;
    asm("{\n\t.reg .b64 A, B, C, D;\n\tmov.b64 A, {%2, %3};\n\tmov.b64 B, {%4, %5};\n\t"
        "mov.b64 C, {%6, %7};\n\tfma.rn.f32x2 D, A, B, C;\n\tmov.b64 {%0, %1}, D;\n\t}"
        : "=f"(r.v.x), "=f"(r.v.y)
        : "f"(a.v.x), "f"(a.v.y), "f"(b.v.x), "f"(b.v.y), "f"(c.v.x), "f"(c.v.y));
    return r;
}
__device__ __forceinline__ F2 recip(F2 a) { return F2(1.0f / a.v.x, 1.0f / a.v.y); }

}  // namespace lbm
