// fixed_sum.cuh -- the fixed summation order of the w quadrature and of the
// weight normalisations: chunk k = t[32k] + ... + t[32k + 31] added left to
// right, then level by level the neighbours (2m, 2m + 1) of the previous
// level added, an unpaired last entry moving up unchanged.  Every FP64
// addition is rounded once (no fused operations), so any implementation of
// this order gives the same double.
//
// Streamed form: terms (or whole chunk sums) arrive in index order; each
// closed chunk is merged with the stacked sums of the same size, as in a
// binary counter.  The stack then holds complete subtrees of decreasing
// size, and folding it from the top, last + previous, ..., reproduces the
// level-by-level pairing with its unpaired entries moving up.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ucp {

constexpr int kSumChunk = 32;

struct FixedSum {
    double stk[40];
    int top = 0;
    int64_t chunks = 0;
    double cur = 0.0;
    int in = 0;

    __device__ __forceinline__ void push_chunk(double s) {
        int64_t n = ++chunks;
        while ((n & 1) == 0) {
            s = __dadd_rn(stk[--top], s);
            n >>= 1;
        }
        stk[top++] = s;
    }
    __device__ __forceinline__ void add(double t) {
        cur = __dadd_rn(cur, t);
        if (++in == kSumChunk) {
            push_chunk(cur);
            cur = 0.0;
            in = 0;
        }
    }
    __device__ __forceinline__ double result() {
        if (in) {
            push_chunk(cur);
            cur = 0.0;
            in = 0;
        }
        if (top == 0) return 0.0;
        double r = stk[top - 1];
        for (int k = top - 2; k >= 0; --k) r = __dadd_rn(stk[k], r);
        return r;
    }
};

// Number of chunks of n terms.
__host__ __device__ inline int64_t sum_chunks(int64_t n) {
    return (n + kSumChunk - 1) / kSumChunk;
}

}  // namespace ucp
