// bench_fp64_probe.cu -- issue rate of FP64 / FP32 FMA and of CUDA math-library
// calls on this GPU (independent chains, full occupancy).  Standalone program:
// python bench_fp64_probe.py builds and runs it.
#include <cstdio>
#include <cuda_runtime.h>

#include "fv_device.cuh"
#define CK(x) do{cudaError_t e=(x); if(e!=cudaSuccess){printf("ERR %s line %d: %s\n",#x,__LINE__,cudaGetErrorString(e)); return 1;}}while(0)
constexpr int ITER=1024;
__global__ void k_dfma(double* out, double b, double c){ double a0=threadIdx.x*1e-3,a1=a0+1,a2=a0+2,a3=a0+3,a4=a0+4,a5=a0+5,a6=a0+6,a7=a0+7;
 for(int i=0;i<ITER;i++){a0=fma(a0,b,c);a1=fma(a1,b,c);a2=fma(a2,b,c);a3=fma(a3,b,c);a4=fma(a4,b,c);a5=fma(a5,b,c);a6=fma(a6,b,c);a7=fma(a7,b,c);}
 out[blockIdx.x*blockDim.x+threadIdx.x]=a0+a1+a2+a3+a4+a5+a6+a7;}
__global__ void k_ffma(float* out, float b, float c){ float a0=threadIdx.x*1e-3f,a1=a0+1,a2=a0+2,a3=a0+3,a4=a0+4,a5=a0+5,a6=a0+6,a7=a0+7;
 for(int i=0;i<ITER;i++){a0=fmaf(a0,b,c);a1=fmaf(a1,b,c);a2=fmaf(a2,b,c);a3=fmaf(a3,b,c);a4=fmaf(a4,b,c);a5=fmaf(a5,b,c);a6=fmaf(a6,b,c);a7=fmaf(a7,b,c);}
 out[blockIdx.x*blockDim.x+threadIdx.x]=a0+a1+a2+a3+a4+a5+a6+a7;}
template<int F> __global__ void k_fn64(double* out, double x0, double dx){ double acc=0; double x=x0+threadIdx.x*1e-6;
 for(int i=0;i<64;i++){ double y;
   if(F==0) y=exp(x); else if(F==1) y=log(x); else if(F==2) y=erfcx(x); else if(F==3) y=erfc(x); else if(F==4) y=1.0/x; else if(F==5) y=sqrt(x); else if (F==6) y=normcdfinv(x*0.1); else if (F==7) y=expm1(x);
   else if(F==8) y=fvd::erfcx64(x); else if(F==9) y=fvd::log64(x); else if(F==10) y=(double)(float)x; else if(F==11) y=3.0/x;
   else if(F==12) y=fvd::exp64(x); else y=log1p(x);
   acc+=y; x+=dx; }
 out[blockIdx.x*blockDim.x+threadIdx.x]=acc;}
template<int F> __global__ void k_fn32(float* out, float x0, float dx){ float acc=0; float x=x0+threadIdx.x*1e-6f;
 for(int i=0;i<256;i++){ float y;
   if(F==0) y=expf(x); else if(F==1) y=logf(x); else if(F==2) y=erfcxf(x); else if(F==3) y=erfcf(x); else if(F==4) y=__fdividef(1.0f,x); else if(F==5) y=sqrtf(x); else if(F==6) y=normcdfinvf(x*0.1f); else y=__expf(x);
   acc+=y; x+=dx; }
 out[blockIdx.x*blockDim.x+threadIdx.x]=acc;}
int main(){
 cudaDeviceProp p; CK(cudaGetDeviceProperties(&p,0)); int clk=0; cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0);
 printf("%s SMs=%d clock(kHz)=%d\n",p.name,p.multiProcessorCount,clk);
 int blocks=p.multiProcessorCount*8, threads=256; size_t n=(size_t)blocks*threads;
 double* d; float* f; CK(cudaMalloc(&d,n*8)); CK(cudaMalloc(&f,n*4));
 cudaEvent_t a,b; cudaEventCreate(&a); cudaEventCreate(&b); float ms;
 auto T=[&](const char* name, double ops, auto launch){ launch(); cudaDeviceSynchronize(); cudaEventRecord(a); for(int r=0;r<5;r++) launch(); cudaEventRecord(b); cudaEventSynchronize(b); cudaEventElapsedTime(&ms,a,b); ms/=5;
   printf("%-12s %9.3f ms  %10.3f Gop/s  %8.3f op/clk/SM (at %d MHz nominal)\n",name,ms,ops/ms*1e-6, ops/(ms*1e-3)/(p.multiProcessorCount*(clk*1e3)), clk/1000); };
 double fmaops=(double)n*ITER*8;
 T("dfma",fmaops,[&]{k_dfma<<<blocks,threads>>>(d,1.0000001,1e-7);});
 T("ffma",fmaops,[&]{k_ffma<<<blocks,threads>>>(f,1.0000001f,1e-7f);});
 double f64ops=(double)n*64, f32ops=(double)n*256;
 T("exp64",f64ops,[&]{k_fn64<0><<<blocks,threads>>>(d,-3.0,1e-3);});
 T("log64",f64ops,[&]{k_fn64<1><<<blocks,threads>>>(d,0.5,1e-3);});
 T("erfcx64",f64ops,[&]{k_fn64<2><<<blocks,threads>>>(d,0.3,1e-2);});
 T("erfc64",f64ops,[&]{k_fn64<3><<<blocks,threads>>>(d,0.3,1e-2);});
 T("rcp64",f64ops,[&]{k_fn64<4><<<blocks,threads>>>(d,0.5,1e-3);});
 T("sqrt64",f64ops,[&]{k_fn64<5><<<blocks,threads>>>(d,0.5,1e-3);});
 T("ncdfinv64",f64ops,[&]{k_fn64<6><<<blocks,threads>>>(d,0.1,1e-3);});
 T("expm1_64",f64ops,[&]{k_fn64<7><<<blocks,threads>>>(d,-0.3,1e-3);});
 T("erfcx64_lib",f64ops,[&]{k_fn64<8><<<blocks,threads>>>(d,0.3,1e-2);});
 T("log64_lib",f64ops,[&]{k_fn64<9><<<blocks,threads>>>(d,0.5,1e-3);});
 T("cvt_f64_f32",f64ops,[&]{k_fn64<10><<<blocks,threads>>>(d,0.5,1e-3);});
 T("div64",f64ops,[&]{k_fn64<11><<<blocks,threads>>>(d,0.5,1e-3);});
 T("exp64_lib",f64ops,[&]{k_fn64<12><<<blocks,threads>>>(d,-3.0,1e-3);});
 T("log1p64",f64ops,[&]{k_fn64<13><<<blocks,threads>>>(d,-0.3,1e-2);});
 T("expf",f32ops,[&]{k_fn32<0><<<blocks,threads>>>(f,-3.0f,1e-3f);});
 T("logf",f32ops,[&]{k_fn32<1><<<blocks,threads>>>(f,0.5f,1e-3f);});
 T("erfcxf",f32ops,[&]{k_fn32<2><<<blocks,threads>>>(f,0.3f,1e-2f);});
 T("erfcf",f32ops,[&]{k_fn32<3><<<blocks,threads>>>(f,0.3f,1e-2f);});
 T("fdividef",f32ops,[&]{k_fn32<4><<<blocks,threads>>>(f,0.5f,1e-3f);});
 T("sqrtf",f32ops,[&]{k_fn32<5><<<blocks,threads>>>(f,0.5f,1e-3f);});
 T("ncdfinvf",f32ops,[&]{k_fn32<6><<<blocks,threads>>>(f,0.1f,1e-3f);});
 T("__expf",f32ops,[&]{k_fn32<7><<<blocks,threads>>>(f,-3.0f,1e-3f);});
 CK(cudaGetLastError());
 printf("OK\n"); return 0;}
