// rt_scan.cu -- exclusive prefix sum of int32 counts (cell lists, reverse lists, per-hop
// requests and receiver segments).  Three kernels: per-block scan, a single-block scan of
// the block totals, and the add-back.  `d_len` (optional) is a device-side element count;
// the scan covers only the entries before it (the output beyond it is left as it was), so a
// launch sized for a capacity scans the live part without a host round trip.
#include "rt_internal.cuh"

#define SCAN_BLOCK 1024

__device__ __forceinline__ int block_excl_scan(int v, int *sh, int *total) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(FULLMASK, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) sh[w] = incl;
    __syncthreads();
    if (w == 0) {
        int s = lane < (blockDim.x >> 5) ? sh[lane] : 0;
        int si = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(FULLMASK, si, o);
            if (lane >= o) si += t;
        }
        sh[lane] = si - s;
        if (lane == 31) sh[32] = si;
    }
    __syncthreads();
    int r = incl - v + sh[w];
    *total = sh[32];
    __syncthreads();
    return r;
}

__global__ void k_scan_blocks(const int *in, int *out, long long n, const int *d_len,
                              int *btot) {
    __shared__ int sh[33];
    long long len = d_len ? (long long)*d_len : n;
    if (len > n) len = n;
    long long b0 = (long long)blockIdx.x * SCAN_BLOCK;
    if (b0 >= len) {   // the whole block lies beyond the live part
        if (threadIdx.x == 0) btot[blockIdx.x] = 0;
        return;
    }
    long long i = b0 + threadIdx.x;
    int v = (i < len) ? in[i] : 0;
    int tot;
    int r = block_excl_scan(v, sh, &tot);
    if (i < len) out[i] = r;
    if (threadIdx.x == 0) btot[blockIdx.x] = tot;
}

__global__ void k_scan_totals(int *btot, long long nblocks, const int *d_len, int *d_total) {
    __shared__ int sh[33];
    int carry = 0;
    if (d_len) {
        long long lb = ((long long)*d_len + SCAN_BLOCK - 1) / SCAN_BLOCK;
        if (lb < nblocks) nblocks = lb;
    }
    for (long long base = 0; base < nblocks; base += SCAN_BLOCK) {
        long long i = base + threadIdx.x;
        int v = i < nblocks ? btot[i] : 0;
        int tot;
        int r = block_excl_scan(v, sh, &tot);
        if (i < nblocks) btot[i] = r + carry;
        carry += tot;
    }
    if (threadIdx.x == 0 && d_total) *d_total = carry;
}

__global__ void k_scan_add(int *out, long long n, const int *d_len, const int *btot) {
    long long len = d_len ? (long long)*d_len : n;
    if (len > n) len = n;
    long long i = (long long)blockIdx.x * SCAN_BLOCK + threadIdx.x;
    if (i < len) out[i] += btot[blockIdx.x];
}

// tmp: block-total scratch of at least scan_tmp_n ints (default: the context's); two scans in
// flight at once need two.  n never exceeds what rt_create sized scan_tmp_n for.
void rt_scan_exclusive(rt_ctx *c, const int *in, int *out, long long n, const int *d_len,
                       int *d_total, cudaStream_t st, int *tmp) {
    long long nb = (n + SCAN_BLOCK - 1) / SCAN_BLOCK;
    if (nb < 1) nb = 1;
    if (!tmp) tmp = c->scan_tmp;
    k_scan_blocks<<<(unsigned)nb, SCAN_BLOCK, 0, st>>>(in, out, n, d_len, tmp);
    k_scan_totals<<<1, SCAN_BLOCK, 0, st>>>(tmp, nb, d_len, d_total);
    k_scan_add<<<(unsigned)nb, SCAN_BLOCK, 0, st>>>(out, n, d_len, tmp);
}
