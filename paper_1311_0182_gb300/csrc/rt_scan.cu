// rt_scan.cu -- exclusive prefix sum of int32 counts (cell lists, reverse lists, per-hop
// requests and receiver segments).  `d_len` (optional) is a device-side element count; the
// scan covers only the entries before it (the output beyond it is left as it was), so a
// launch made for a capacity scans the live part without a host round trip.
#include "rt_internal.cuh"

#define SCAN_BLOCK 1024

template <typename T>
__device__ __forceinline__ T block_excl_scan(T v, T *sh, T *total) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T t = __shfl_up_sync(FULLMASK, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) sh[w] = incl;
    __syncthreads();
    if (w == 0) {
        T s = lane < (int)(blockDim.x >> 5) ? sh[lane] : T(0);
        T si = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T t = __shfl_up_sync(FULLMASK, si, o);
            if (lane >= o) si += t;
        }
        sh[lane] = si - s;
        if (lane == 31) sh[32] = si;
    }
    __syncthreads();
    T r = incl - v + sh[w];
    *total = sh[32];
    __syncthreads();
    return r;
}

// Two kernels on a fixed grid of SCAN_NB blocks: block b owns one contiguous range of the
// live part; the first kernel sums each range, the second scans it in tiles of SCAN_BLOCK,
// starting from the sum of the ranges before it.  No launch is sized by the capacity.
#define SCAN_NB RT_SCAN_NB

__device__ __forceinline__ void scan_range(long long len, long long &b0, long long &b1) {
    long long per = (len + SCAN_NB - 1) / SCAN_NB;
    per = (per + SCAN_BLOCK - 1) / SCAN_BLOCK * SCAN_BLOCK;   // whole tiles per block
    b0 = (long long)blockIdx.x * per;
    b1 = b0 + per < len ? b0 + per : len;
}

__device__ __forceinline__ long long scan_len(long long n, const int *d_len) {
    long long len = d_len ? (long long)*d_len : n;
    return len < n ? len : n;
}

__global__ void __launch_bounds__(SCAN_BLOCK) k_scan_sum(const int *in, long long n,
                                                         const int *d_len, int *btot) {
    __shared__ int sh[33];
    long long b0, b1;
    scan_range(scan_len(n, d_len), b0, b1);
    int v = 0;
    for (long long i = b0 + threadIdx.x; i < b1; i += SCAN_BLOCK) v += in[i];
    int tot;
    block_excl_scan(v, sh, &tot);
    if (threadIdx.x == 0) btot[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(SCAN_BLOCK) k_scan_fin(const int *in, int *out, long long n,
                                                         const int *d_len, const int *btot,
                                                         int *d_total) {
    __shared__ int sh[33];
    long long b0, b1;
    scan_range(scan_len(n, d_len), b0, b1);
    // the sum of the ranges before this block (and of all of them, for the total)
    int before = 0, all = 0;
    for (int k = threadIdx.x; k < SCAN_NB; k += SCAN_BLOCK) {
        int t = btot[k];
        all += t;
        if (k < (int)blockIdx.x) before += t;
    }
    int tb, ta;
    block_excl_scan(before, sh, &tb);
    block_excl_scan(all, sh, &ta);
    if (blockIdx.x == 0 && threadIdx.x == 0 && d_total) *d_total = ta;
    int carry = tb;
    for (long long base = b0; base < b1; base += SCAN_BLOCK) {
        long long i = base + threadIdx.x;
        int v = i < b1 ? in[i] : 0;
        int tot;
        int r = block_excl_scan(v, sh, &tot);
        if (i < b1) out[i] = carry + r;
        carry += tot;
    }
}

// tmp: block-total scratch of at least SCAN_NB ints (default: the context's); two scans in
// flight at once need two.
void rt_scan_exclusive(rt_ctx *c, const int *in, int *out, long long n, const int *d_len,
                       int *d_total, cudaStream_t st, int *tmp) {
    if (!tmp) tmp = c->scan_tmp;
    k_scan_sum<<<SCAN_NB, SCAN_BLOCK, 0, st>>>(in, n, d_len, tmp);
    k_scan_fin<<<SCAN_NB, SCAN_BLOCK, 0, st>>>(in, out, n, d_len, tmp, d_total);
}

// The same scan into 64-bit offsets (the per-cell candidate lists, whose total can pass 2^31):
// counts are int32, sums and offsets int64; no device-side length.
__global__ void __launch_bounds__(SCAN_BLOCK) k_scan64_sum(const int *in, long long n,
                                                           long long *btot) {
    __shared__ long long sh[33];
    long long b0, b1;
    scan_range(n, b0, b1);
    long long v = 0;
    for (long long i = b0 + threadIdx.x; i < b1; i += SCAN_BLOCK) v += in[i];
    long long tot;
    block_excl_scan(v, sh, &tot);
    if (threadIdx.x == 0) btot[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(SCAN_BLOCK) k_scan64_fin(const int *in, long long *out,
                                                           long long n, const long long *btot) {
    __shared__ long long sh[33];
    long long b0, b1;
    scan_range(n, b0, b1);
    long long before = 0;
    for (int k = threadIdx.x; k < (int)blockIdx.x; k += SCAN_BLOCK) before += btot[k];
    long long tb;
    block_excl_scan(before, sh, &tb);
    long long carry = tb;
    for (long long base = b0; base < b1; base += SCAN_BLOCK) {
        long long i = base + threadIdx.x;
        long long v = i < b1 ? (long long)in[i] : 0;
        long long tot;
        long long r = block_excl_scan(v, sh, &tot);
        if (i < b1) out[i] = carry + r;
        carry += tot;
    }
}

// tmp: SCAN_NB 64-bit block totals (device)
void rt_scan_exclusive64(const int *in, long long *out, long long n, long long *tmp,
                         cudaStream_t st) {
    k_scan64_sum<<<SCAN_NB, SCAN_BLOCK, 0, st>>>(in, n, tmp);
    k_scan64_fin<<<SCAN_NB, SCAN_BLOCK, 0, st>>>(in, out, n, tmp);
}
