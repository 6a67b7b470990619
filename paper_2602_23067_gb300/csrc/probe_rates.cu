// probe_rates.cu -- microbenchmarks behind the design's rate arguments
// (built into libgcmprobe.so, separate from the product library).
//
// Each kernel runs one CTA per SM and times its own loop with the SM clock
// (clock64 after a barrier on both sides), so rates come out per clock per
// SM without knowing the clock frequency:
//   * integer issue rates of the instructions the table engine and the
//     bitsliced engine are made of: 3-input logic (lop3), byte permute
//     (prmt), funnel shift (shf), multiply-add (mad.lo), add;
//   * shared-memory lookups in the fused kernel's own addressing: 4-byte
//     round-table lookups with a per-lane bank column (conflict-free by
//     construction), the same lookups with unreplicated random addresses,
//     and 16-byte GHASH-table lookups with the lane-rotated byte positions;
//   * random 4-byte gathers through the texture and constant caches, alone
//     and interleaved with shared-memory lookups (do the paths add up?);
//   * the 1-bit tensor-core product (mma.sync m16n8k256, AND + popcount),
//     the natural GF(2) multiply, in dependent and independent chains;
//   * host-memory access over the CPU-GPU link: a kernel reading or writing
//     page-locked host memory, and the copy engines on the same buffers.
// Every loop is bounded; no kernel waits on another.
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <cuda_runtime.h>

namespace {

constexpr int CHAINS = 8;

__device__ __forceinline__ uint32_t op_lop3(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t r;
    asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
    return r;
}
__device__ __forceinline__ uint32_t op_prmt(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t r;
    asm volatile("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
    return r;
}
__device__ __forceinline__ uint32_t op_shf(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t r;
    asm volatile("shf.l.wrap.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
    return r;
}
__device__ __forceinline__ uint32_t op_mad(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t r;
    asm volatile("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
    return r;
}
__device__ __forceinline__ uint32_t op_add(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t r;
    asm volatile("add.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    (void)c;
    return r;
}

template <int OP>
__device__ __forceinline__ uint32_t apply(uint32_t a, uint32_t b, uint32_t c)
{
    if (OP == 0) return op_lop3(a, b, c);
    if (OP == 1) return op_prmt(a, b, c);
    if (OP == 2) return op_shf(a, b, c);
    if (OP == 3) return op_mad(a, b, c);
    return op_add(a, b, c);
}

template <int OP>
__global__ void alu_kernel(int iters, uint32_t *sink, unsigned long long *cycles)
{
    uint32_t a[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; c++) a[c] = threadIdx.x * 0x9E3779B9u + c;
    const uint32_t b = 0x01234567u ^ blockIdx.x, k = (OP == 1) ? 0x5410u : 0x3u + (blockIdx.x & 1);
    __syncthreads();
    const unsigned long long t0 = clock64();
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < CHAINS; c++) a[c] = apply<OP>(a[c], b, k);
    }
    __syncthreads();
    const unsigned long long t1 = clock64();
    uint32_t x = 0;
#pragma unroll
    for (int c = 0; c < CHAINS; c++) x ^= a[c];
    if (x == 0x12345678u) sink[threadIdx.x] = x;  // keeps the chains alive
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

// Round-table lookups in the table engine's own instruction mix: a 4-word
// state per thread goes through AES-like rounds, each column of a round the
// XOR of four lookups (byte r of word c + r selects the row) and a key word.
// MODE 0: the fused kernel's layout, 128 KiB of rows [T_even x 32 lanes |
// T_odd x 32 lanes], address = byte permute of (row byte, lane column), so
// every lane reads its own bank; MODE 1: the four 1 KiB tables unreplicated
// (address = table * 1024 + row * 4), so banks collide by chance.  16
// lookups per round; the round's four columns are independent, the rounds
// are not (as in AES).
template <int MODE>
__global__ void lds32_kernel(int iters, uint32_t *sink, unsigned long long *cycles)
{
    extern __shared__ uint8_t tb[];
    for (int i = threadIdx.x; i < 32768; i += blockDim.x)
        reinterpret_cast<uint32_t *>(tb)[i] = (uint32_t)i * 2654435761u;
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t cA = lane * 4u, cB = 128u + lane * 4u;
    const uint8_t *t01 = tb, *t23 = tb + 65536;
    uint32_t s0 = threadIdx.x * 0x9E3779B9u, s1 = s0 ^ 0x12345678u, s2 = s0 * 3u, s3 = ~s0;
    const uint32_t k = 0x0F1E2D3Cu ^ blockIdx.x;
#define PL(t, w, B, c) (*reinterpret_cast<const uint32_t *>((t) + __byte_perm((w), (c), 0x5504u | ((B) << 4))))
#define RL(T, w, B) (*reinterpret_cast<const uint32_t *>(tb + (T) * 1024u + ((((w) >> (8 * (B))) & 0xFFu) << 2)))
    const unsigned long long t0 = clock64();
    for (int i = 0; i < iters; i++) {
        uint32_t n0, n1, n2, n3;
        if (MODE == 0) {
            n0 = PL(t01, s0, 0, cA) ^ PL(t01, s1, 1, cB) ^ PL(t23, s2, 2, cA) ^ PL(t23, s3, 3, cB) ^ k;
            n1 = PL(t01, s1, 0, cA) ^ PL(t01, s2, 1, cB) ^ PL(t23, s3, 2, cA) ^ PL(t23, s0, 3, cB) ^ k;
            n2 = PL(t01, s2, 0, cA) ^ PL(t01, s3, 1, cB) ^ PL(t23, s0, 2, cA) ^ PL(t23, s1, 3, cB) ^ k;
            n3 = PL(t01, s3, 0, cA) ^ PL(t01, s0, 1, cB) ^ PL(t23, s1, 2, cA) ^ PL(t23, s2, 3, cB) ^ k;
        } else {
            n0 = RL(0, s0, 0) ^ RL(1, s1, 1) ^ RL(2, s2, 2) ^ RL(3, s3, 3) ^ k;
            n1 = RL(0, s1, 0) ^ RL(1, s2, 1) ^ RL(2, s3, 2) ^ RL(3, s0, 3) ^ k;
            n2 = RL(0, s2, 0) ^ RL(1, s3, 1) ^ RL(2, s0, 2) ^ RL(3, s1, 3) ^ k;
            n3 = RL(0, s3, 0) ^ RL(1, s0, 1) ^ RL(2, s1, 2) ^ RL(3, s2, 3) ^ k;
        }
        s0 = n0; s1 = n1; s2 = n2; s3 = n3;
    }
#undef PL
#undef RL
    __syncthreads();
    const unsigned long long t1 = clock64();
    if ((s0 ^ s1 ^ s2 ^ s3) == 0x12345678u) sink[threadIdx.x] = s0;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

// GHASH-table lookups: 256 rows of 16 positions x 16 bytes (64 KiB); lane l
// reads position (l + step) mod 8 (+ 8 for the second half), so the 8 lanes
// of a quarter-warp touch 8 distinct 16-byte bank groups.
__global__ void lds128_kernel(int iters, uint32_t *sink, unsigned long long *cycles)
{
    extern __shared__ uint4 gt[];
    for (int i = threadIdx.x; i < 4096; i += blockDim.x)
        gt[i] = make_uint4(i * 2654435761u, i * 40503u, i * 9973u, i ^ 0x5A5A5A5Au);
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31;
    uint4 acc[2];
    acc[0] = make_uint4(threadIdx.x, 1u, 2u, 3u);
    acc[1] = make_uint4(threadIdx.x * 3u, 5u, 7u, 11u);
    const unsigned long long t0 = clock64();
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int s = 0; s < 8; s++) {
#pragma unroll
            for (int c = 0; c < 2; c++) {
                const uint32_t pos = ((lane + s) & 7u) + 8u * c;
                const uint4 v = gt[((acc[c].x & 0xFFu) << 4) | pos];
                acc[c].x ^= v.x + (uint32_t)s;
                acc[c].y ^= v.y;
                acc[c].z ^= v.z;
                acc[c].w ^= v.w;
            }
        }
    }
    __syncthreads();
    const unsigned long long t1 = clock64();
    if ((acc[0].x ^ acc[0].y ^ acc[1].z ^ acc[1].w) == 0x12345678u) sink[threadIdx.x] = acc[0].x;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

// 1-bit tensor-core product: D = popc(A AND B) + C, m16n8k256, CH independent
// accumulators per warp (CH = 1: a dependent chain, for the latency).
template <int CH>
__global__ void mma_b1_kernel(int iters, uint32_t *sink, unsigned long long *cycles)
{
    uint32_t a[4] = {threadIdx.x, threadIdx.x * 3u, 0xFFFFFFFFu, 0x0F0F0F0Fu};
    uint32_t b[2] = {0x33333333u ^ threadIdx.x, 0x55555555u};
    int32_t d[CH][4];
#pragma unroll
    for (int c = 0; c < CH; c++)
#pragma unroll
        for (int k = 0; k < 4; k++) d[c][k] = c + k;
    __syncthreads();
    const unsigned long long t0 = clock64();
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < CH; c++)
            asm volatile(
                "mma.sync.aligned.m16n8k256.row.col.s32.b1.b1.s32.and.popc "
                "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
                : "+r"(d[c][0]), "+r"(d[c][1]), "+r"(d[c][2]), "+r"(d[c][3])
                : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    }
    __syncthreads();
    const unsigned long long t1 = clock64();
    int32_t x = 0;
#pragma unroll
    for (int c = 0; c < CH; c++) x ^= d[c][0] ^ d[c][3];
    if (x == 0x12345678) sink[threadIdx.x] = (uint32_t)x;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

// Random 4-byte gathers through other paths than the shared-memory pipe:
// PATH 0 texture fetches (tex1Dfetch over a 64 KiB linear texture), PATH 1
// divergent constant-cache loads (16 KiB __constant__ table), PATH 2 both
// interleaved with conflict-free shared-memory lookups (RATIO shared
// lookups per texture fetch), to see whether the paths add up.
__constant__ uint32_t c_tab[4096];

template <int PATH, int RATIO>
__global__ void gather_kernel(cudaTextureObject_t tex, int iters, uint32_t *sink, unsigned long long *cycles)
{
    extern __shared__ uint32_t tab[];
    if (PATH == 2) {
        for (int i = threadIdx.x; i < 16384; i += blockDim.x) tab[i] = (uint32_t)i * 2654435761u;
    }
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31;
    constexpr int S = 8;
    uint32_t a[S], acc[S], b[S];
#pragma unroll
    for (int c = 0; c < S; c++) {
        a[c] = (threadIdx.x * 2654435761u) ^ (c * 0x9E3779B9u);
        b[c] = a[c] & 0x3FC0u;
        acc[c] = 0u;
    }
    const unsigned long long t0 = clock64();
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < S; c++) {
            if (PATH == 0 || PATH == 2) acc[c] += tex1Dfetch<uint32_t>(tex, (int)(a[c] & 0x3FFFu));
            if (PATH == 1) acc[c] += c_tab[a[c] & 0xFFFu];
            a[c] += 2654435761u;
            if (PATH == 2) {
#pragma unroll
                for (int k = 0; k < RATIO; k++) {
                    acc[c] += tab[(b[c] & 0x3FC0u) | lane | ((k & 1) << 5)];
                    b[c] += 0x40u * 37u;
                }
            }
        }
    }
    __syncthreads();
    const unsigned long long t1 = clock64();
    uint32_t x = 0;
#pragma unroll
    for (int c = 0; c < S; c++) x ^= acc[c] ^ a[c] ^ b[c];
    if (x == 0x12345678u) sink[threadIdx.x] = x;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

// Host memory through the link: 16-byte loads (xor-reduced) or stores over
// a grid-stride range.
__global__ void host_read_kernel(const uint4 *p, size_t n, uint4 *sink)
{
    uint4 acc = make_uint4(0u, 0u, 0u, 0u);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const uint4 v = __ldcs(p + i);
        acc.x ^= v.x; acc.y ^= v.y; acc.z ^= v.z; acc.w ^= v.w;
    }
    if ((acc.x ^ acc.y ^ acc.z ^ acc.w) == 0x12345678u) sink[0] = acc;
}

__global__ void host_write_kernel(uint4 *p, size_t n)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        __stcs(p + i, make_uint4((uint32_t)i, 1u, 2u, 3u));
}

int g_err_line = 0;
#define CK(x)                                  \
    do {                                       \
        cudaError_t e_ = (x);                  \
        if (e_ != cudaSuccess) {               \
            g_err_line = __LINE__;             \
            return (int)e_;                    \
        }                                      \
    } while (0)

// Runs a cycle-timed kernel on one CTA per SM; returns the median over SMs
// of the loop's cycles.
template <typename F>
int run_cycles(F launch, int sms, double *median_cycles)
{
    unsigned long long *d_cyc = nullptr;
    uint32_t *d_sink = nullptr;
    CK(cudaMalloc(&d_cyc, sizeof(unsigned long long) * sms));
    CK(cudaMalloc(&d_sink, 4096 * sizeof(uint32_t)));
    launch(d_sink, d_cyc);  // warm-up
    CK(cudaGetLastError());
    CK(cudaDeviceSynchronize());
    launch(d_sink, d_cyc);
    CK(cudaGetLastError());
    CK(cudaDeviceSynchronize());
    unsigned long long h[1024];
    CK(cudaMemcpy(h, d_cyc, sizeof(unsigned long long) * sms, cudaMemcpyDeviceToHost));
    // insertion sort (at most a few hundred entries)
    for (int i = 1; i < sms; i++) {
        unsigned long long v = h[i];
        int j = i - 1;
        while (j >= 0 && h[j] > v) {
            h[j + 1] = h[j];
            j--;
        }
        h[j + 1] = v;
    }
    *median_cycles = (double)h[sms / 2];
    cudaFree(d_cyc);
    cudaFree(d_sink);
    return 0;
}

// A 256-byte S-box held in registers across the warp: lane l keeps bytes
// 8l..8l+7 in two words; looking up byte x fetches both words of lane x / 8
// with two shuffles and selects byte x mod 8 with a byte permute.
__device__ __forceinline__ uint32_t shfl_lookup(uint32_t x, uint32_t lo, uint32_t hi)
{
    const int src = (int)((x >> 3) & 31u);
    const uint32_t a = __shfl_sync(0xFFFFFFFFu, lo, src);
    const uint32_t b = __shfl_sync(0xFFFFFFFFu, hi, src);
    return __byte_perm(a, b, x & 7u) & 0xFFu;
}

// MIX = 0: shuffle lookups alone (4 independent chains per thread).  MIX > 0:
// every iteration is one AES-like round on the replicated round tables (16
// shared lookups, as in lds32_kernel MODE 0) plus MIX shuffle lookups, to
// see whether shuffles take capacity from the shared-memory pipe.
template <int MIX>
__global__ void shfl_kernel(int iters, uint32_t *sink, unsigned long long *cycles)
{
    extern __shared__ uint8_t tb[];
    if (MIX > 0)
        for (int i = threadIdx.x; i < 32768; i += blockDim.x)
            reinterpret_cast<uint32_t *>(tb)[i] = (uint32_t)i * 2654435761u;
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t lo = lane * 0x9E3779B9u, hi = lane * 0x7F4A7C15u;
    const uint32_t cA = lane * 4u, cB = 128u + lane * 4u;
    const uint8_t *t01 = tb, *t23 = tb + 65536;
    uint32_t s0 = threadIdx.x * 0x9E3779B9u, s1 = s0 ^ 0x12345678u, s2 = s0 * 3u, s3 = ~s0;
    const uint32_t k = 0x0F1E2D3Cu ^ blockIdx.x;
    uint32_t x[4];
#pragma unroll
    for (int c = 0; c < 4; c++) x[c] = threadIdx.x * 7919u + 104729u * c;
#define PL(t, w, B, c) (*reinterpret_cast<const uint32_t *>((t) + __byte_perm((w), (c), 0x5504u | ((B) << 4))))
    const unsigned long long t0 = clock64();
    for (int i = 0; i < iters; i++) {
        if (MIX > 0) {
            const uint32_t n0 = PL(t01, s0, 0, cA) ^ PL(t01, s1, 1, cB) ^ PL(t23, s2, 2, cA) ^ PL(t23, s3, 3, cB) ^ k;
            const uint32_t n1 = PL(t01, s1, 0, cA) ^ PL(t01, s2, 1, cB) ^ PL(t23, s3, 2, cA) ^ PL(t23, s0, 3, cB) ^ k;
            const uint32_t n2 = PL(t01, s2, 0, cA) ^ PL(t01, s3, 1, cB) ^ PL(t23, s0, 2, cA) ^ PL(t23, s1, 3, cB) ^ k;
            const uint32_t n3 = PL(t01, s3, 0, cA) ^ PL(t01, s0, 1, cB) ^ PL(t23, s1, 2, cA) ^ PL(t23, s2, 3, cB) ^ k;
            s0 = n0; s1 = n1; s2 = n2; s3 = n3;
        }
#pragma unroll
        for (int c = 0; c < (MIX > 0 ? MIX : 4); c++) x[c & 3] = shfl_lookup(x[c & 3], lo, hi) + (x[c & 3] >> 8) + (uint32_t)i;
    }
#undef PL
    __syncthreads();
    const unsigned long long t1 = clock64();
    if ((s0 ^ s1 ^ s2 ^ s3 ^ x[0] ^ x[1] ^ x[2] ^ x[3]) == 0x12345678u) sink[threadIdx.x] = s0;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

}  // namespace

extern "C" {

int probe_last_error_line(void) { return g_err_line; }

// Integer issue rate: op 0 lop3, 1 prmt, 2 shf, 3 mad.lo, 4 add.  Writes
// thread-instructions per clock per SM (threads x iters x chains / cycles).
int probe_alu(int op, int threads, int iters, double *per_clk_per_sm)
{
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (sms > 1024 || threads <= 0 || threads > 1024 || iters <= 0) return -1;
    double cyc = 0;
    auto launch = [&](uint32_t *sink, unsigned long long *c) {
        switch (op) {
        case 0: alu_kernel<0><<<sms, threads>>>(iters, sink, c); break;
        case 1: alu_kernel<1><<<sms, threads>>>(iters, sink, c); break;
        case 2: alu_kernel<2><<<sms, threads>>>(iters, sink, c); break;
        case 3: alu_kernel<3><<<sms, threads>>>(iters, sink, c); break;
        default: alu_kernel<4><<<sms, threads>>>(iters, sink, c); break;
        }
    };
    int rc = run_cycles(launch, sms, &cyc);
    if (rc) return rc;
    *per_clk_per_sm = (double)threads * iters * CHAINS / cyc;
    return 0;
}

// Shared-memory lookups per clock per SM (lanes, i.e. individual lookups):
// kind 0 AES-like rounds on the replicated round tables (conflict-free), 1
// the same rounds on unreplicated tables, 2 16-byte GHASH-table lookups with
// rotated positions.
int probe_lds(int kind, int threads, int iters, double *lookups_per_clk_per_sm)
{
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (sms > 1024 || threads <= 0 || threads > 1024 || iters <= 0 || kind < 0 || kind > 2) return -1;
    const int smem = 65536, smem32 = 131072;
    CK(cudaFuncSetAttribute(lds32_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem32));
    CK(cudaFuncSetAttribute(lds32_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem32));
    CK(cudaFuncSetAttribute(lds128_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    double cyc = 0;
    auto launch = [&](uint32_t *sink, unsigned long long *c) {
        if (kind == 0) lds32_kernel<0><<<sms, threads, smem32>>>(iters, sink, c);
        else if (kind == 1) lds32_kernel<1><<<sms, threads, smem32>>>(iters, sink, c);
        else lds128_kernel<<<sms, threads, smem>>>(iters, sink, c);
    };
    int rc = run_cycles(launch, sms, &cyc);
    if (rc) return rc;
    const double per_iter = 16.0;  // lookups per thread per iteration (one round, or 8 x 2 GHASH lookups)
    *lookups_per_clk_per_sm = (double)threads * iters * per_iter / cyc;
    return 0;
}

// Random 4-byte gathers per clock per SM through other paths: kind 0
// texture fetches, 1 divergent constant-cache loads, 2 texture fetches
// interleaved with 8 conflict-free shared-memory lookups each (the result
// counts both kinds of lookup), 3 the same with 24 shared lookups each.
int probe_gather(int kind, int threads, int iters, double *lookups_per_clk_per_sm)
{
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (sms > 1024 || threads <= 0 || threads > 1024 || iters <= 0 || kind < 0 || kind > 3) return -1;
    uint32_t *d_tab = nullptr;
    CK(cudaMalloc(&d_tab, 65536));
    uint32_t h[16384];
    for (int i = 0; i < 16384; i++) h[i] = (uint32_t)i * 2246822519u;
    CK(cudaMemcpy(d_tab, h, 65536, cudaMemcpyHostToDevice));
    CK(cudaMemcpyToSymbol(c_tab, h, sizeof(uint32_t) * 4096));
    cudaResourceDesc rd;
    memset(&rd, 0, sizeof(rd));
    rd.resType = cudaResourceTypeLinear;
    rd.res.linear.devPtr = d_tab;
    rd.res.linear.desc = cudaCreateChannelDesc<uint32_t>();
    rd.res.linear.sizeInBytes = 65536;
    cudaTextureDesc td;
    memset(&td, 0, sizeof(td));
    td.readMode = cudaReadModeElementType;
    cudaTextureObject_t tex = 0;
    CK(cudaCreateTextureObject(&tex, &rd, &td, nullptr));
    const int smem = 65536;
    CK(cudaFuncSetAttribute(gather_kernel<2, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    CK(cudaFuncSetAttribute(gather_kernel<2, 24>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    double cyc = 0;
    auto launch = [&](uint32_t *sink, unsigned long long *c) {
        if (kind == 0) gather_kernel<0, 0><<<sms, threads>>>(tex, iters, sink, c);
        else if (kind == 1) gather_kernel<1, 0><<<sms, threads>>>(tex, iters, sink, c);
        else if (kind == 2) gather_kernel<2, 8><<<sms, threads, smem>>>(tex, iters, sink, c);
        else gather_kernel<2, 24><<<sms, threads, smem>>>(tex, iters, sink, c);
    };
    int rc = run_cycles(launch, sms, &cyc);
    cudaDestroyTextureObject(tex);
    cudaFree(d_tab);
    if (rc) return rc;
    const double per_iter = (kind == 2) ? 8.0 * 9 : (kind == 3) ? 8.0 * 25 : 8.0;
    *lookups_per_clk_per_sm = (double)threads * iters * per_iter / cyc;
    return 0;
}

// Warp-shuffle S-box lookups (two shuffles and a byte permute each):
// out[0] shared-memory round-table lookups and out[1] shuffle lookups, per
// clock per SM.  mix 0 runs shuffle lookups alone; mix 4, 8 or 16 adds that
// many per AES-like round of 16 shared lookups.
int probe_shfl(int mix, int threads, int iters, double out[2])
{
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (sms > 1024 || threads <= 0 || threads > 1024 || (threads & 31) || iters <= 0) return -1;
    if (mix != 0 && mix != 4 && mix != 8 && mix != 16) return -1;
    const int smem32 = 131072;
    CK(cudaFuncSetAttribute(shfl_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem32));
    CK(cudaFuncSetAttribute(shfl_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem32));
    CK(cudaFuncSetAttribute(shfl_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem32));
    double cyc = 0;
    auto launch = [&](uint32_t *sink, unsigned long long *c) {
        if (mix == 0) shfl_kernel<0><<<sms, threads>>>(iters, sink, c);
        else if (mix == 4) shfl_kernel<4><<<sms, threads, smem32>>>(iters, sink, c);
        else if (mix == 8) shfl_kernel<8><<<sms, threads, smem32>>>(iters, sink, c);
        else shfl_kernel<16><<<sms, threads, smem32>>>(iters, sink, c);
    };
    int rc = run_cycles(launch, sms, &cyc);
    if (rc) return rc;
    out[0] = mix ? (double)threads * iters * 16.0 / cyc : 0.0;
    out[1] = (double)threads * iters * (mix ? mix : 4) / cyc;
    return 0;
}

// 1-bit mma.sync (m16n8k256, AND + popcount): warp-level instructions per
// clock per SM with `chains` independent accumulators per warp (1 or 4).
int probe_mma_b1(int chains, int threads, int iters, double *mma_per_clk_per_sm)
{
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (sms > 1024 || threads <= 0 || threads > 1024 || (threads & 31) || iters <= 0) return -1;
    double cyc = 0;
    auto launch = [&](uint32_t *sink, unsigned long long *c) {
        if (chains == 1) mma_b1_kernel<1><<<sms, threads>>>(iters, sink, c);
        else mma_b1_kernel<4><<<sms, threads>>>(iters, sink, c);
    };
    int rc = run_cycles(launch, sms, &cyc);
    if (rc) return rc;
    *mma_per_clk_per_sm = (double)(threads / 32) * iters * (chains == 1 ? 1 : 4) / cyc;
    return 0;
}

// Host memory over the link, GB/s: out[0] kernel read of page-locked memory,
// out[1] kernel write of page-locked memory, out[2] copy engine host to
// device, out[3] device to host, out[4] and out[5] both directions at once
// (each way), out[6] kernel read of ordinary (pageable) host memory, or -1
// when the device cannot access pageable memory.  `bytes` per transfer.
int probe_host(size_t bytes, int reps, double out[7])
{
    int dev = 0, sms = 0, pageable = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CK(cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, dev));
    bytes &= ~(size_t)15;
    if (bytes == 0 || reps <= 0) return -1;
    const size_t n = bytes / 16;
    uint8_t *h_a = nullptr, *h_b = nullptr, *d_a = nullptr, *d_b = nullptr;
    uint4 *d_sink = nullptr;
    CK(cudaHostAlloc(&h_a, bytes, cudaHostAllocDefault));
    CK(cudaHostAlloc(&h_b, bytes, cudaHostAllocDefault));
    CK(cudaMalloc(&d_a, bytes));
    CK(cudaMalloc(&d_b, bytes));
    CK(cudaMalloc(&d_sink, 16));
    for (size_t i = 0; i < bytes; i += 4096) h_a[i] = (uint8_t)i, h_b[i] = (uint8_t)(i >> 12);
    cudaStream_t s1, s2;
    CK(cudaStreamCreateWithFlags(&s1, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking));
    cudaEvent_t e0, e1, e2, e3;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaEventCreate(&e2));
    CK(cudaEventCreate(&e3));
    float ms = 0;
    const int grid = sms * 4, block = 512;
    auto timed = [&](auto fn, double *gbs) -> int {
        fn();  // warm-up
        CK(cudaStreamSynchronize(s1));
        CK(cudaEventRecord(e0, s1));
        for (int r = 0; r < reps; r++) fn();
        CK(cudaEventRecord(e1, s1));
        CK(cudaEventSynchronize(e1));
        CK(cudaEventElapsedTime(&ms, e0, e1));
        *gbs = (double)bytes * reps / (ms * 1e-3) / 1e9;
        return 0;
    };
    int rc;
    rc = timed([&] { host_read_kernel<<<grid, block, 0, s1>>>(reinterpret_cast<const uint4 *>(h_a), n, d_sink); },
               &out[0]);
    if (rc) return rc;
    rc = timed([&] { host_write_kernel<<<grid, block, 0, s1>>>(reinterpret_cast<uint4 *>(h_b), n); }, &out[1]);
    if (rc) return rc;
    rc = timed([&] { cudaMemcpyAsync(d_a, h_a, bytes, cudaMemcpyHostToDevice, s1); }, &out[2]);
    if (rc) return rc;
    rc = timed([&] { cudaMemcpyAsync(h_b, d_b, bytes, cudaMemcpyDeviceToHost, s1); }, &out[3]);
    if (rc) return rc;
    // both directions at once, on two streams
    CK(cudaDeviceSynchronize());
    CK(cudaEventRecord(e0, s1));
    CK(cudaEventRecord(e2, s2));
    for (int r = 0; r < reps; r++) {
        CK(cudaMemcpyAsync(d_a, h_a, bytes, cudaMemcpyHostToDevice, s1));
        CK(cudaMemcpyAsync(h_b, d_b, bytes, cudaMemcpyDeviceToHost, s2));
    }
    CK(cudaEventRecord(e1, s1));
    CK(cudaEventRecord(e3, s2));
    CK(cudaDeviceSynchronize());
    CK(cudaEventElapsedTime(&ms, e0, e1));
    out[4] = (double)bytes * reps / (ms * 1e-3) / 1e9;
    CK(cudaEventElapsedTime(&ms, e2, e3));
    out[5] = (double)bytes * reps / (ms * 1e-3) / 1e9;
    out[6] = -1.0;
    if (pageable) {
        uint8_t *m = static_cast<uint8_t *>(malloc(bytes));
        if (m) {
            for (size_t i = 0; i < bytes; i += 4096) m[i] = (uint8_t)i;  // touch every page
            rc = timed([&] { host_read_kernel<<<grid, block, 0, s1>>>(reinterpret_cast<const uint4 *>(m), n, d_sink); },
                       &out[6]);
            free(m);
            if (rc) return rc;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(e2);
    cudaEventDestroy(e3);
    cudaStreamDestroy(s1);
    cudaStreamDestroy(s2);
    cudaFreeHost(h_a);
    cudaFreeHost(h_b);
    cudaFree(d_a);
    cudaFree(d_b);
    cudaFree(d_sink);
    return 0;
}

}  // extern "C"
