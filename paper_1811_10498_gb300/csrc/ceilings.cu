// Hardware ceilings that decide the scan kernels' design (bench.py --suite ceilings):
//   * store bandwidth for 1 GiB of int32 output: memset, 16-byte stores from grids of
//     several shapes (with and without an evict-first L2 hint), 32-byte stores, and TMA
//     bulk stores of a zero tile in shared memory issued by one lane per warp;
//   * random 4-byte lookup rates: global memory over buffers of 128 KB to 512 MB (L1, L2
//     and HBM resident), local shared memory, and distributed shared memory of thread-block
//     clusters of 2 to 16 CTAs (each CTA holds 128 KB; every lookup goes to a random CTA
//     of the cluster).
// Prints one JSON line per measurement. Every index is masked to its buffer's size.
#include <cstdio>
#include <cstdint>
#include <cstdlib>
#include <vector>
#include <algorithm>
#include <cuda_runtime.h>

#define CK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { printf("{\"error\": \"%s\", \"line\": %d}\n", cudaGetErrorString(e_), __LINE__); exit(1);} } while (0)

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__global__ void store_plain(int4 *out, int64_t n4)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = make_int4(0, 0, 0, 0);
}

__global__ void store_hint(int4 *out, int64_t n4)
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x)
        asm volatile("st.global.L2::cache_hint.v4.b32 [%0], {%1, %1, %1, %1}, %2;" ::"l"(out + i), "r"(0), "l"(pol) : "memory");
}

// 32-byte stores (st.global.v8.b32), one per thread-iteration.
__global__ void store_v8(int4 *out, int64_t n8)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n8; i += (int64_t)gridDim.x * blockDim.x)
        asm volatile("st.global.v8.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1};" ::"l"(out + 2 * i), "r"(0) : "memory");
}

// One elected lane per warp issues bulk stores of `chunk` bytes from a zero buffer.
template <bool HINT>
__global__ void store_bulk(uint8_t *out, int64_t n_chunks, int chunk, int depth)
{
    extern __shared__ __align__(128) uint8_t zb[];
    for (int i = threadIdx.x * 16; i < chunk; i += blockDim.x * 16) *reinterpret_cast<int4 *>(zb + i) = make_int4(0, 0, 0, 0);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    if (lane == 0) {
        int inflight = 0;
        for (int64_t c = w; c < n_chunks; c += warps) {
            if (HINT)
                asm volatile("cp.async.bulk.global.shared::cta.bulk_group.L2::cache_hint [%0], [%1], %2, %3;" ::"l"(out + c * chunk),
                             "r"(smem_addr(zb)), "r"(chunk), "l"(pol) : "memory");
            else
                asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(out + c * chunk),
                             "r"(smem_addr(zb)), "r"(chunk) : "memory");
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
            if (++inflight >= depth) {
                asm volatile("cp.async.bulk.wait_group.read 4;" ::: "memory");
                inflight = 4;
            }
        }
        asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    }
}

__device__ __forceinline__ uint32_t hash32(uint32_t x)
{
    x ^= x >> 16; x *= 0x7feb352du; x ^= x >> 15; x *= 0x846ca68bu; x ^= x >> 16;
    return x;
}

__global__ void l2_lookup(const uint32_t *__restrict__ buf, uint32_t mask, int R, uint32_t *out)
{
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t acc = 0, h = hash32(tid * 0x9E3779B9u + 1u);
#pragma unroll 16
    for (int i = 0; i < R; i++) {
        h = h * 1664525u + 1013904223u;
        acc ^= __ldg(buf + (hash32(h) & mask));
    }
    out[tid] = acc;
}

__global__ void smem_lookup(int R, uint32_t *out)
{
    extern __shared__ uint32_t s[];
    for (int i = threadIdx.x; i < 32768; i += blockDim.x) s[i] = i * 2654435761u;
    __syncthreads();
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t acc = 0, h = hash32(tid * 0x9E3779B9u + 1u);
#pragma unroll 16
    for (int i = 0; i < R; i++) {
        h = h * 1664525u + 1013904223u;
        acc ^= s[hash32(h) & 32767u];
    }
    out[tid] = acc;
}

__device__ __forceinline__ void cluster_sync_all()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__global__ void dsmem_lookup(int R, uint32_t cs_mask, uint32_t *out)
{
    extern __shared__ uint32_t s[];
    for (int i = threadIdx.x; i < 32768; i += blockDim.x) s[i] = i * 2654435761u;
    cluster_sync_all();
    const uint32_t base = smem_addr(s);
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t acc = 0, h = hash32(tid * 0x9E3779B9u + 1u);
#pragma unroll 16
    for (int i = 0; i < R; i++) {
        h = h * 1664525u + 1013904223u;
        const uint32_t x = hash32(h);
        const uint32_t rank = (x >> 15) & cs_mask;
        uint32_t ra, v;
        asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(base + 4u * (x & 32767u)), "r"(rank));
        asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(ra) : "memory");
        acc ^= v;
    }
    cluster_sync_all();
    out[tid] = acc;
}

template <typename F>
static float time_ms(F f, int reps = 10)
{
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    for (int i = 0; i < 3; i++) f();
    CK(cudaDeviceSynchronize());
    std::vector<float> ts;
    for (int i = 0; i < reps; i++) {
        CK(cudaEventRecord(a));
        f();
        CK(cudaEventRecord(b));
        CK(cudaEventSynchronize(b));
        float ms;
        CK(cudaEventElapsedTime(&ms, a, b));
        ts.push_back(ms);
    }
    std::sort(ts.begin(), ts.end());
    return ts[ts.size() / 2];
}

int main()
{
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0));
    printf("{\"sms\": %d}\n", sms);
    const int64_t n = 268435456;   // int32 elements = 1 GiB
    const int64_t bytes = n * 4;
    uint8_t *out;
    CK(cudaMalloc(&out, bytes));
    auto gbs = [&](float ms) { return bytes / (ms * 1e-3) / 1e9; };

    float ms = time_ms([&] { cudaMemsetAsync(out, 0, bytes); });
    printf("{\"test\": \"store\", \"kind\": \"memset\", \"ms\": %.4f, \"gbs\": %.0f}\n", ms, gbs(ms));
    for (int blocks_per_sm : {2, 4, 8, 16}) {
        ms = time_ms([&] { store_plain<<<sms * blocks_per_sm, 256>>>((int4 *)out, n / 4); });
        printf("{\"test\": \"store\", \"kind\": \"v4\", \"blocks_per_sm\": %d, \"threads\": 256, \"ms\": %.4f, \"gbs\": %.0f}\n", blocks_per_sm, ms, gbs(ms));
    }
    ms = time_ms([&] { store_hint<<<sms * 8, 256>>>((int4 *)out, n / 4); });
    printf("{\"test\": \"store\", \"kind\": \"v4 evict_first\", \"blocks_per_sm\": 8, \"threads\": 256, \"ms\": %.4f, \"gbs\": %.0f}\n", ms, gbs(ms));
    ms = time_ms([&] { store_hint<<<sms, 1024>>>((int4 *)out, n / 4); });
    printf("{\"test\": \"store\", \"kind\": \"v4 evict_first\", \"blocks_per_sm\": 1, \"threads\": 1024, \"ms\": %.4f, \"gbs\": %.0f}\n", ms, gbs(ms));
    for (int blocks_per_sm : {2, 8}) {
        ms = time_ms([&] { store_v8<<<sms * blocks_per_sm, 256>>>((int4 *)out, n / 8); });
        printf("{\"test\": \"store\", \"kind\": \"v8\", \"blocks_per_sm\": %d, \"threads\": 256, \"ms\": %.4f, \"gbs\": %.0f}\n", blocks_per_sm, ms, gbs(ms));
    }
    for (int chunk : {4096, 16384}) {
        CK(cudaFuncSetAttribute(store_bulk<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, chunk));
        CK(cudaFuncSetAttribute(store_bulk<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, chunk));
        for (int warps : {1, 4, 31}) {
            for (int depth : {8, 16}) {
                const int64_t nch = bytes / chunk;
                ms = time_ms([&] { store_bulk<false><<<sms, 32 * warps, chunk>>>(out, nch, chunk, depth); });
                printf("{\"test\": \"store\", \"kind\": \"bulk\", \"chunk\": %d, \"warps\": %d, \"depth\": %d, \"hint\": 0, \"ms\": %.4f, \"gbs\": %.0f}\n", chunk, warps, depth, ms, gbs(ms));
                ms = time_ms([&] { store_bulk<true><<<sms, 32 * warps, chunk>>>(out, nch, chunk, depth); });
                printf("{\"test\": \"store\", \"kind\": \"bulk\", \"chunk\": %d, \"warps\": %d, \"depth\": %d, \"hint\": 1, \"ms\": %.4f, \"gbs\": %.0f}\n", chunk, warps, depth, ms, gbs(ms));
            }
        }
    }
    CK(cudaGetLastError());

    // lookups
    uint32_t *buf;
    const int64_t buf_bytes = 512ll << 20;
    CK(cudaMalloc(&buf, buf_bytes));
    CK(cudaMemset(buf, 0x5a, buf_bytes));
    uint32_t *res;
    const int max_threads = sms * 2048;
    CK(cudaMalloc(&res, (size_t)max_threads * 4));
    const int R = 256;
    for (int64_t fb : {128ll << 10, 2ll << 20, 32ll << 20, 512ll << 20}) {
        const uint32_t mask = (uint32_t)(fb / 4 - 1);
        ms = time_ms([&] { l2_lookup<<<sms * 2, 1024>>>(buf, mask, R, res); });
        const double loads = (double)sms * 2048 * R;
        printf("{\"test\": \"lookup\", \"kind\": \"global\", \"kb\": %lld, \"ms\": %.4f, \"g_loads_s\": %.1f}\n", (long long)(fb >> 10), ms, loads / (ms * 1e-3) / 1e9);
    }
    CK(cudaFuncSetAttribute(smem_lookup, cudaFuncAttributeMaxDynamicSharedMemorySize, 131072));
    ms = time_ms([&] { smem_lookup<<<sms, 1024, 131072>>>(R, res); });
    printf("{\"test\": \"lookup\", \"kind\": \"shared\", \"kb\": 128, \"ms\": %.4f, \"g_loads_s\": %.1f}\n", ms, (double)sms * 1024 * R / (ms * 1e-3) / 1e9);

    CK(cudaFuncSetAttribute(dsmem_lookup, cudaFuncAttributeMaxDynamicSharedMemorySize, 131072));
    CK(cudaFuncSetAttribute(dsmem_lookup, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    for (int cs : {2, 4, 8, 16}) {
        cudaLaunchConfig_t lc = {};
        lc.blockDim = dim3(1024);
        lc.dynamicSmemBytes = 131072;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cs;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        lc.attrs = attr;
        lc.numAttrs = 1;
        lc.gridDim = dim3(cs);
        int clusters = 0;
        cudaError_t e = cudaOccupancyMaxActiveClusters(&clusters, dsmem_lookup, &lc);
        if (e != cudaSuccess || clusters <= 0) {
            printf("{\"test\": \"lookup\", \"kind\": \"dsmem\", \"cluster\": %d, \"unavailable\": \"%s\", \"clusters\": %d}\n", cs, cudaGetErrorString(e), clusters);
            cudaGetLastError();
            continue;
        }
        lc.gridDim = dim3(clusters * cs);
        const int blocks = clusters * cs;
        ms = time_ms([&] { cudaLaunchKernelEx(&lc, dsmem_lookup, R, (uint32_t)(cs - 1), res); });
        CK(cudaGetLastError());
        printf("{\"test\": \"lookup\", \"kind\": \"dsmem\", \"cluster\": %d, \"clusters\": %d, \"ctas\": %d, \"ms\": %.4f, \"g_loads_s\": %.1f}\n",
               cs, clusters, blocks, ms, (double)blocks * 1024 * R / (ms * 1e-3) / 1e9);
    }
    CK(cudaDeviceSynchronize());
    printf("{\"done\": 1}\n");
    return 0;
}
