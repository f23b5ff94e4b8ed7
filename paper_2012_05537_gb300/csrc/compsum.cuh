// Error-free transformations and compensated sums in FP32 and FP64, shared by the step
// kernels' compensated moment sums (the moments of Eq. moments to about one rounding).
#pragma once

namespace sllbm {

// Rounded arithmetic that the compiler may neither contract into an FMA nor reorder (the
// error-free transformations below rely on every operation being rounded on its own).
__device__ __forceinline__ float add_rn(float x, float y) { return __fadd_rn(x, y); }
__device__ __forceinline__ float sub_rn(float x, float y) { return __fsub_rn(x, y); }
__device__ __forceinline__ float mul_rn(float x, float y) { return __fmul_rn(x, y); }
__device__ __forceinline__ double add_rn(double x, double y) { return __dadd_rn(x, y); }
__device__ __forceinline__ double sub_rn(double x, double y) { return __dsub_rn(x, y); }
__device__ __forceinline__ double mul_rn(double x, double y) { return __dmul_rn(x, y); }

// Compensated summation: s holds the rounded running sum and c the exact rounding errors of
// its additions (Knuth's branch-free two-sum: t = s + x, z = t - s, error (s - (t - z)) +
// (x - z)), so that s + c carries the sum to about one rounding of the result whatever the
// number of terms.  Products enter with the rounding error of the product itself recovered
// by an FMA (two-product), so a sum of products is compensated as well.
template <typename C>
struct CompSum {
    C s = C(0), c = C(0);
    __device__ __forceinline__ void add(C x) {
        const C t = add_rn(s, x);
        const C z = sub_rn(t, s);
        c = add_rn(c, add_rn(sub_rn(s, sub_rn(t, z)), sub_rn(x, z)));
        s = t;
    }
    __device__ __forceinline__ void add_prod(C x, C y) {
        const C p = mul_rn(x, y);
        add(p);
        c = add_rn(c, fma(x, y, -p));  // the product's own rounding error, exactly
    }
    // another compensated partial sum (its rounded sum and its error term)
    __device__ __forceinline__ void add_partial(C ps, C pc) {
        add(ps);
        c = add_rn(c, pc);
    }
    __device__ __forceinline__ C value() const { return add_rn(s, c); }
};

}  // namespace sllbm
