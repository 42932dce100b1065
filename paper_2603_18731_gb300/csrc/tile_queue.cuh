// Device tile queue of the packed products.
//
// The rows of many (operator, subspace) pairs are cut into tiles (a fixed
// number of rows of one pair); tile t belongs to the last pair whose first
// tile is <= t.  A persistent grid (the blocks that fit on the SMs at once)
// serves every tile of the queue: each block claims the next tile with one
// atomic increment, loads the pair's parameters into shared memory when the
// pair changes, evaluates the tile's rows and claims again until the tiles
// run out.  No block waits for another: a claim never blocks, and the last
// block to leave resets the queue (claim and exit counters to zero), so the
// next launch on the same stream finds it ready.  That makes a launch
// independent of the pair count and sizes -- the grid and the kernel
// arguments stay the same when the pairs change -- so a CUDA graph captured
// once replays for any membership written into the queue's device block.
#pragma once

#include <cstdint>

namespace qsd {

struct TileQueue {
    int32_t n;                   // pairs
    int32_t pad;
    int64_t tiles;               // total tiles
    unsigned long long next;     // claim counter (0 between launches)
    unsigned long long exited;   // blocks that have left (0 between launches)
};

// Pair of tile t: binary search over the pairs' first tiles (ascending, t0[0] = 0).
__device__ __forceinline__ int tile_pair(const int64_t *__restrict__ t0, int n, int64_t t) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (t0[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Persistent loop over the queue.  P: the per-pair parameter record (a
// multiple of 4 bytes), copied to `sp` in shared memory; body(sp, pair,
// tile_in_pair) evaluates one tile with the whole block.  Every block-level
// branch depends only on shared values, so all threads take it together.
template <typename P, typename Body>
__device__ __forceinline__ void run_tile_queue(const P *__restrict__ params, const int64_t *__restrict__ t0,
                                               TileQueue *q, P &sp, Body body) {
    static_assert(sizeof(P) % 4 == 0, "parameter copy by words");
    __shared__ long long s_tile;
    __shared__ int s_pair;
    const int n = q->n;
    const long long tiles = q->tiles;
    int cur = -1;
    for (;;) {
        if (threadIdx.x == 0) {
            const long long t = (long long)atomicAdd(&q->next, 1ull);
            s_tile = t;
            if (t < tiles) s_pair = tile_pair(t0, n, t);
        }
        __syncthreads();
        const long long t = s_tile;
        if (t >= tiles) break;
        const int pr = s_pair;
        if (pr != cur) {
            const uint32_t *src = reinterpret_cast<const uint32_t *>(params + pr);
            uint32_t *dst = reinterpret_cast<uint32_t *>(&sp);
            for (int i = threadIdx.x; i < (int)(sizeof(P) / 4); i += blockDim.x) dst[i] = __ldg(src + i);
            __syncthreads();
            cur = pr;
        }
        body(sp, pr, t - t0[pr]);
        __syncthreads();  // sp and the claim are rewritten next round
    }
    // the last block out resets the queue: every other block has made its
    // final claim before counting itself out
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&q->exited, 1ull) == (unsigned long long)gridDim.x - 1) {
            q->next = 0;
            q->exited = 0;
            __threadfence();
        }
    }
}

}  // namespace qsd
