// host_link.cu -- device -> host bandwidth of the two ways a result can
// reach host memory on this machine: copy-engine copies into pinned memory
// (cudaMemcpyAsync, one stream and two streams at once) and SM stores into
// pinned host memory mapped into the device's address space (the emit
// kernel's store pattern: 32-byte streaming stores, consecutive lanes on
// consecutive addresses).  Also host -> device copies, for the inputs.
// CUDA events, best of 5, 4 GiB per transfer.
// Standalone: nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o host_link
//   host_link.cu && ./host_link
#include <cstdint>
#include <cstdio>

#include <cuda_runtime.h>

#define CK(x)                                                                        \
    do {                                                                             \
        cudaError_t e_ = (x);                                                        \
        if (e_ != cudaSuccess) {                                                     \
            printf("CUDA error %s at line %d\n", cudaGetErrorString(e_), __LINE__);  \
            return 1;                                                                \
        }                                                                            \
    } while (0)

// every thread writes 32 contiguous bytes per step (one v4.b64 store)
__global__ void store32(unsigned long long *p, int64_t n4) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
         i += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long *q = p + 4 * i;
        asm volatile("st.global.cs.v4.b64 [%0], {%1, %2, %3, %4};" ::"l"(q), "l"((unsigned long long)i),
                     "l"((unsigned long long)i + 1), "l"((unsigned long long)i + 2),
                     "l"((unsigned long long)i + 3) : "memory");
    }
}

int main() {
    const size_t bytes = 4ull << 30;
    void *dev = nullptr, *host = nullptr, *dev_mapped = nullptr;
    CK(cudaMalloc(&dev, bytes));
    CK(cudaMemset(dev, 1, bytes));
    CK(cudaHostAlloc(&host, bytes, cudaHostAllocMapped));
    CK(cudaHostGetDevicePointer(&dev_mapped, host, 0));
    cudaStream_t s1, s2;
    CK(cudaStreamCreateWithFlags(&s1, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking));
    cudaEvent_t a, b, j;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    CK(cudaEventCreate(&j));
    auto run = [&](const char *name, auto launch) {
        for (int w = 0; w < 2; w++) launch();
        CK(cudaDeviceSynchronize());
        float best = 1e30f;
        for (int r = 0; r < 5; r++) {
            cudaEventRecord(a, s1);
            cudaStreamWaitEvent(s2, a, 0);
            launch();
            cudaEventRecord(j, s2);
            cudaStreamWaitEvent(s1, j, 0);
            cudaEventRecord(b, s1);
            cudaEventSynchronize(b);
            float ms;
            cudaEventElapsedTime(&ms, a, b);
            if (ms < best) best = ms;
        }
        printf("%-40s %8.3f ms %8.1f GB/s\n", name, best, bytes / best / 1e6);
        return 0;
    };
    run("D2H copy, one stream", [&] { cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, s1); });
    run("D2H copy, two streams", [&] {
        cudaMemcpyAsync(host, dev, bytes / 2, cudaMemcpyDeviceToHost, s1);
        cudaMemcpyAsync((char *)host + bytes / 2, (char *)dev + bytes / 2, bytes / 2,
                        cudaMemcpyDeviceToHost, s2);
    });
    run("H2D copy, one stream", [&] { cudaMemcpyAsync(dev, host, bytes, cudaMemcpyHostToDevice, s1); });
    const int64_t n4 = (int64_t)(bytes / 32);
    run("SM stores into mapped pinned memory", [&] {
        store32<<<152 * 8, 256, 0, s1>>>((unsigned long long *)dev_mapped, n4);
    });
    run("SM stores into device memory", [&] {
        store32<<<152 * 8, 256, 0, s1>>>((unsigned long long *)dev, n4);
    });
    CK(cudaGetLastError());
    CK(cudaDeviceSynchronize());
    // the stores really reached host memory
    const unsigned long long *h = (const unsigned long long *)host;
    printf("host check: %llu %llu %llu\n", h[0], h[5], h[4 * (n4 - 1) + 3]);
    cudaFreeHost(host);
    cudaFree(dev);
    return 0;
}
