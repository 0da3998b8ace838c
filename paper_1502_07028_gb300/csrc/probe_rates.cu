// probe_rates.cu -- standalone throughput probe of one GPU: FP64 and FP32 FMA,
// FP64 and FP32 division, and shared-memory 64-bit load bandwidth.  These
// are the ALU and shared-memory peaks the cluster kernels' rooflines are read
// against (the Householder reduction is bound by the FP32 pipe and shared
// memory, the plain FP64 path by the FP64 pipe).  Not part of the library.
//
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o probe_rates probe_rates.cu && ./probe_rates
//
// All indexing stays inside the buffers allocated below; no waits, no atomics.
#include <cstdio>
#include <cuda_runtime.h>
#define CK(x) do{cudaError_t e=(x); if(e!=cudaSuccess){printf("err %s line %d\n",cudaGetErrorString(e),__LINE__); return 1;}}while(0)

template<typename T> __global__ void fma_k(T* out, int iters, T a, T b){
  T x0=threadIdx.x, x1=x0+1, x2=x0+2, x3=x0+3, x4=x0+4, x5=x0+5, x6=x0+6, x7=x0+7;
  for(int i=0;i<iters;i++){
    x0=x0*a+b; x1=x1*a+b; x2=x2*a+b; x3=x3*a+b; x4=x4*a+b; x5=x5*a+b; x6=x6*a+b; x7=x7*a+b;
  }
  out[blockIdx.x*blockDim.x+threadIdx.x]=x0+x1+x2+x3+x4+x5+x6+x7;
}
template<typename T> __global__ void div_k(T* out, int iters, T a){
  T x0=threadIdx.x+1, x1=x0+1, x2=x0+2, x3=x0+3;
  for(int i=0;i<iters;i++){ x0=a/x0+1; x1=a/x1+1; x2=a/x2+1; x3=a/x3+1; }
  out[blockIdx.x*blockDim.x+threadIdx.x]=x0+x1+x2+x3;
}
__global__ void fastdiv_k(float* out, int iters, float a){
  float x0=threadIdx.x+1, x1=x0+1, x2=x0+2, x3=x0+3;
  for(int i=0;i<iters;i++){ x0=__fdividef(a,x0)+1; x1=__fdividef(a,x1)+1; x2=__fdividef(a,x2)+1; x3=__fdividef(a,x3)+1; }
  out[blockIdx.x*blockDim.x+threadIdx.x]=x0+x1+x2+x3;
}
__global__ void smem_k(float* out, int iters){
  __shared__ float2 s[4096];
  for(int i=threadIdx.x;i<4096;i+=blockDim.x) s[i]=make_float2(i,i);
  __syncthreads();
  float2 acc=make_float2(0,0);
  int idx=threadIdx.x;
  for(int i=0;i<iters;i++){
    float2 v=s[(idx+i*32)&4095]; acc.x+=v.x; acc.y+=v.y;
  }
  out[blockIdx.x*blockDim.x+threadIdx.x]=acc.x+acc.y;
}
int main(){
  int dev=0; cudaDeviceProp p; CK(cudaGetDeviceProperties(&p,dev));
  int sms=p.multiProcessorCount; printf("SMs %d smemPerBlockOptin %zu\n",sms,p.sharedMemPerBlockOptin);
  int blocks=sms*4, threads=256; size_t N=(size_t)blocks*threads;
  double* dd; float* ff; CK(cudaMalloc(&dd,N*8)); CK(cudaMalloc(&ff,N*4));
  cudaEvent_t a,b; cudaEventCreate(&a); cudaEventCreate(&b); float ms;
  // FP64 FMA
  for(int rep=0;rep<2;rep++){
    int it=1<<12; cudaEventRecord(a); fma_k<double><<<blocks,threads>>>(dd,it,0.999,0.001); cudaEventRecord(b); CK(cudaEventSynchronize(b)); cudaEventElapsedTime(&ms,a,b);
    if(rep) printf("FP64 FMA: %.3f TFLOP/s\n", 2.0*8*it*N/ms/1e9);
  }
  for(int rep=0;rep<2;rep++){
    int it=1<<16; cudaEventRecord(a); fma_k<float><<<blocks,threads>>>(ff,it,0.999f,0.001f); cudaEventRecord(b); CK(cudaEventSynchronize(b)); cudaEventElapsedTime(&ms,a,b);
    if(rep) printf("FP32 FMA: %.3f TFLOP/s\n", 2.0*8*it*N/ms/1e9);
  }
  for(int rep=0;rep<2;rep++){
    int it=1<<10; cudaEventRecord(a); div_k<double><<<blocks,threads>>>(dd,it,3.0); cudaEventRecord(b); CK(cudaEventSynchronize(b)); cudaEventElapsedTime(&ms,a,b);
    if(rep) printf("FP64 div: %.3f Gdiv/s\n", 4.0*it*N/ms/1e6);
  }
  for(int rep=0;rep<2;rep++){
    int it=1<<14; cudaEventRecord(a); div_k<float><<<blocks,threads>>>(ff,it,3.0f); cudaEventRecord(b); CK(cudaEventSynchronize(b)); cudaEventElapsedTime(&ms,a,b);
    if(rep) printf("FP32 div (IEEE): %.3f Gdiv/s\n", 4.0*it*N/ms/1e6);
  }
  for(int rep=0;rep<2;rep++){
    int it=1<<14; cudaEventRecord(a); fastdiv_k<<<blocks,threads>>>(ff,it,3.0f); cudaEventRecord(b); CK(cudaEventSynchronize(b)); cudaEventElapsedTime(&ms,a,b);
    if(rep) printf("FP32 fast div: %.3f Gdiv/s\n", 4.0*it*N/ms/1e6);
  }
  for(int rep=0;rep<2;rep++){
    int it=1<<14; cudaEventRecord(a); smem_k<<<blocks,threads>>>(ff,it); cudaEventRecord(b); CK(cudaEventSynchronize(b)); cudaEventElapsedTime(&ms,a,b);
    if(rep) printf("smem LDS.64: %.3f TB/s\n", 8.0*it*N/ms/1e9);
  }
  CK(cudaGetLastError());
  return 0;
}
