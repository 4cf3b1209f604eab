// Peaks probe for the roofline of FP64-pipe-bound stencils on GB300: FP64 and
// FP32 FMA throughput, cost of masked lanes, DDIV / DSQRT cost, shared-memory
// load rate and kernel-launch latency (stream and CUDA graph).  A standalone
// program, not part of the library: python peaks_probe.py builds and runs it.  Every
// kernel writes only indices below blocks * threads of a 64 MiB buffer.
#include <cstdio>
#include <cuda_runtime.h>
#define CK(x) do{cudaError_t e=(x); if(e!=cudaSuccess){printf("ERR %s @%d: %s\n",#x,__LINE__,cudaGetErrorString(e)); return 1;}}while(0)

template<int CH>
__global__ void dfma_k(double* out, int iters, double a, double b, int active_lanes) {
  int lane = threadIdx.x & 31;
  double x[CH];
  #pragma unroll
  for (int c=0;c<CH;++c) x[c] = threadIdx.x*1e-9 + c;
  if (lane < active_lanes) {
    for (int i=0;i<iters;++i) {
      #pragma unroll
      for (int c=0;c<CH;++c) x[c] = fma(x[c], a, b);
    }
  }
  double s=0;
  #pragma unroll
  for (int c=0;c<CH;++c) s+=x[c];
  if (s == 12345.678) out[blockIdx.x*blockDim.x+threadIdx.x] = s;
}
template<int CH>
__global__ void dadd_k(double* out, int iters, double a) {
  double x[CH];
  #pragma unroll
  for (int c=0;c<CH;++c) x[c] = threadIdx.x*1e-9 + c;
  for (int i=0;i<iters;++i) {
    #pragma unroll
    for (int c=0;c<CH;++c) x[c] = __dadd_rn(x[c], a);
  }
  double s=0;
  #pragma unroll
  for (int c=0;c<CH;++c) s+=x[c];
  if (s == 12345.678) out[blockIdx.x*blockDim.x+threadIdx.x] = s;
}
template<int CH>
__global__ void ddiv_k(double* out, int iters, double a) {
  double x[CH];
  #pragma unroll
  for (int c=0;c<CH;++c) x[c] = 1.0 + threadIdx.x*1e-9 + c;
  for (int i=0;i<iters;++i) {
    #pragma unroll
    for (int c=0;c<CH;++c) x[c] = a / x[c] + 1.0;
  }
  double s=0;
  #pragma unroll
  for (int c=0;c<CH;++c) s+=x[c];
  if (s == 12345.678) out[blockIdx.x*blockDim.x+threadIdx.x] = s;
}
template<int CH>
__global__ void dsqrt_k(double* out, int iters) {
  double x[CH];
  #pragma unroll
  for (int c=0;c<CH;++c) x[c] = 2.0 + threadIdx.x*1e-9 + c;
  for (int i=0;i<iters;++i) {
    #pragma unroll
    for (int c=0;c<CH;++c) x[c] = sqrt(x[c]) + 1.0;
  }
  double s=0;
  #pragma unroll
  for (int c=0;c<CH;++c) s+=x[c];
  if (s == 12345.678) out[blockIdx.x*blockDim.x+threadIdx.x] = s;
}
template<int CH>
__global__ void ffma_k(float* out, int iters, float a, float b) {
  float x[CH];
  #pragma unroll
  for (int c=0;c<CH;++c) x[c] = threadIdx.x*1e-9f + c;
  for (int i=0;i<iters;++i) {
    #pragma unroll
    for (int c=0;c<CH;++c) x[c] = fmaf(x[c], a, b);
  }
  float s=0;
  #pragma unroll
  for (int c=0;c<CH;++c) s+=x[c];
  if (s == 12345.678f) out[blockIdx.x*blockDim.x+threadIdx.x] = s;
}
__global__ void empty_k() {}
// dependent FP64 chain: latency of one DFMA / DADD, one warp per block
__global__ void dfma_lat_k(double* out, int iters, double a, double b) {
  double x = threadIdx.x * 1e-9;
  for (int i = 0; i < iters; ++i) x = fma(x, a, b);
  if (x == 12345.678) out[blockIdx.x * blockDim.x + threadIdx.x] = x;
}
// __syncthreads round trip with 8 warps and no other work
__global__ void bar_k(double* out, int iters) {
  double x = threadIdx.x;
  for (int i = 0; i < iters; ++i) { __syncthreads(); x += 1.0; }
  if (x == 12345.678) out[blockIdx.x * blockDim.x + threadIdx.x] = x;
}
// shared-memory bandwidth: each thread reads 8B words in a strided-free pattern
__global__ void smem_k(double* out, int iters) {
  __shared__ double sm[4096];
  for (int i=threadIdx.x;i<4096;i+=blockDim.x) sm[i]=i;
  __syncthreads();
  double s=0; int idx=threadIdx.x;
  for (int i=0;i<iters;++i) { s += sm[idx]; idx = (idx + blockDim.x) & 4095; s += sm[idx]; idx = (idx + blockDim.x) & 4095; }
  if (s == 12345.678) out[blockIdx.x*blockDim.x+threadIdx.x] = s;
}

int main() {
  int dev=0; cudaDeviceProp p; CK(cudaGetDeviceProperties(&p, dev));
  int clk=0, l2=0; cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev); cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
  int smemOptin=0; cudaDeviceGetAttribute(&smemOptin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  printf("name=%s sms=%d cc=%d.%d clk_khz=%d l2=%d smem_optin=%d smem_per_sm=%zu regs_per_sm=%d\n", p.name, p.multiProcessorCount, p.major, p.minor, clk, l2, smemOptin, p.sharedMemPerMultiprocessor, p.regsPerMultiprocessor);
  int sms = p.multiProcessorCount;
  double* dout; CK(cudaMalloc(&dout, 1<<26));
  cudaEvent_t e0,e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  float ms;
  const int CH=8;
  // DFMA full warps, varying blocks/threads
  int cfgs[][2] = {{1,128},{1,256},{2,256},{4,256},{8,256},{4,512},{8,1024}};
  for (auto& c : cfgs) {
    int blocks = sms*c[0], thr=c[1]; int iters=2000;
    dfma_k<CH><<<blocks,thr>>>(dout, 10, 1.0000001, 1e-7, 32); CK(cudaDeviceSynchronize());
    cudaEventRecord(e0); dfma_k<CH><<<blocks,thr>>>(dout, iters, 1.0000001, 1e-7, 32); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms,e0,e1);
    double ops = (double)blocks*thr*iters*CH;
    printf("DFMA blocks/sm=%d thr=%d : %.3f ms  %.2f Gop/s  %.3f TFLOP/s  ops/clk/SM(at 2070)=%.3f\n", c[0], thr, ms, ops/ms/1e6, 2*ops/ms/1e9, ops/(ms*1e-3)/sms/2.07e9);
  }
  for (int act : {32,16,8,1}) {
    int blocks = sms*4, thr=256; int iters=2000;
    cudaEventRecord(e0); dfma_k<CH><<<blocks,thr>>>(dout, iters, 1.0000001, 1e-7, act); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms,e0,e1);
    double ops = (double)blocks*thr*iters*CH*act/32.0;
    printf("DFMA active_lanes=%d : %.3f ms  lane-ops %.2f Gop/s (warp-instr rate %.2f G/s)\n", act, ms, ops/ms/1e6, ops/act/ms/1e6);
  }
  { int blocks=sms*4, thr=256, iters=2000;
    dadd_k<CH><<<blocks,thr>>>(dout, 10, 1e-7); CK(cudaDeviceSynchronize());
    cudaEventRecord(e0); dadd_k<CH><<<blocks,thr>>>(dout, iters, 1e-7); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms,e0,e1); double ops=(double)blocks*thr*iters*CH;
    printf("DADD : %.3f ms %.2f Gop/s\n", ms, ops/ms/1e6); }
  { int blocks=sms*4, thr=256, iters=200;
    ddiv_k<CH><<<blocks,thr>>>(dout, 10, 0.5); CK(cudaDeviceSynchronize());
    cudaEventRecord(e0); ddiv_k<CH><<<blocks,thr>>>(dout, iters, 0.5); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms,e0,e1); double ops=(double)blocks*thr*iters*CH;
    printf("DDIV(+add) : %.3f ms %.3f Gdiv/s\n", ms, ops/ms/1e6); }
  { int blocks=sms*4, thr=256, iters=200;
    dsqrt_k<CH><<<blocks,thr>>>(dout, 10); CK(cudaDeviceSynchronize());
    cudaEventRecord(e0); dsqrt_k<CH><<<blocks,thr>>>(dout, iters); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms,e0,e1); double ops=(double)blocks*thr*iters*CH;
    printf("DSQRT(+add) : %.3f ms %.3f Gsqrt/s\n", ms, ops/ms/1e6); }
  { int blocks=sms*8, thr=512, iters=20000;
    ffma_k<CH><<<blocks,thr>>>((float*)dout, 10, 1.0000001f, 1e-7f); CK(cudaDeviceSynchronize());
    cudaEventRecord(e0); ffma_k<CH><<<blocks,thr>>>((float*)dout, iters, 1.0000001f, 1e-7f); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms,e0,e1); double ops=(double)blocks*thr*iters*CH;
    printf("FFMA : %.3f ms %.2f TFLOP/s  ops/clk/SM(2070)=%.1f\n", ms, 2*ops/ms/1e9, ops/(ms*1e-3)/sms/2.07e9); }
  { int blocks=sms*8, thr=512, iters=20000;
    smem_k<<<blocks,thr>>>(dout, 10); CK(cudaDeviceSynchronize());
    cudaEventRecord(e0); smem_k<<<blocks,thr>>>(dout, iters); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms,e0,e1); double bytes=(double)blocks*thr*iters*2*8;
    printf("SMEM LDS.64 : %.3f ms %.2f TB/s  B/clk/SM(2070)=%.1f\n", ms, bytes/ms/1e9, bytes/(ms*1e-3)/sms/2.07e9); }
  { int iters = 100000;
    dfma_lat_k<<<sms, 32>>>(dout, 10, 1.0000001, 1e-7); CK(cudaDeviceSynchronize());
    cudaEventRecord(e0); dfma_lat_k<<<sms, 32>>>(dout, iters, 1.0000001, 1e-7); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms,e0,e1);
    printf("DFMA dependent latency (1 warp/SM): %.2f ns = %.1f clk at 2070 MHz\n", ms*1e6/iters, ms*1e6/iters*2.07); }
  { int iters = 100000;
    bar_k<<<sms, 256>>>(dout, 10); CK(cudaDeviceSynchronize());
    cudaEventRecord(e0); bar_k<<<sms, 256>>>(dout, iters); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms,e0,e1);
    printf("__syncthreads + DADD loop (8 warps): %.2f ns = %.1f clk per iteration\n", ms*1e6/iters, ms*1e6/iters*2.07); }
  // launch latency
  { int n=20000; for (int i=0;i<100;++i) empty_k<<<1,32>>>(); CK(cudaDeviceSynchronize());
    cudaEventRecord(e0); for (int i=0;i<n;++i) empty_k<<<1,32>>>(); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms,e0,e1); printf("empty launch (stream, back-to-back): %.3f us\n", ms*1e3/n);
    cudaStream_t s; cudaStreamCreate(&s); cudaGraph_t g; cudaGraphExec_t ge;
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeGlobal)); for (int i=0;i<1000;++i) empty_k<<<152,128,0,s>>>(); CK(cudaStreamEndCapture(s,&g));
    CK(cudaGraphInstantiate(&ge, g, 0)); CK(cudaGraphLaunch(ge, s)); CK(cudaStreamSynchronize(s));
    cudaEventRecord(e0, s); for (int r=0;r<10;++r) cudaGraphLaunch(ge, s); cudaEventRecord(e1, s); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms,e0,e1); printf("empty kernel in graph (152x128): %.3f us/kernel\n", ms*1e3/10000);
    cudaEventRecord(e0, s); for (int i=0;i<n;++i) empty_k<<<152,128,0,s>>>(); cudaEventRecord(e1, s); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms,e0,e1); printf("empty launch 152x128 stream: %.3f us\n", ms*1e3/n);
  }
  printf("done\n");
  return 0;
}
