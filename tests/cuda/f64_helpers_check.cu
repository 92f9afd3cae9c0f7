// Checks the FP64 kernels' exact bit helpers (mp_f64math.cuh) against
// CUDA's own conversions and frexp/ldexp on every input class of their
// domains; prints the mismatch counts and exits non-zero on any.
#include <cstdio>

#include "mp_f64math.cuh"

using namespace mp;

__device__ __forceinline__ unsigned long long mix64(unsigned long long x)
{
    x += 0x9e3779b97f4a7c15ULL;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ULL;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebULL;
    return x ^ (x >> 31);
}

__global__ void check(unsigned long long* bad, unsigned long long n)
{
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        // f2d_pos: every non-negative FP32 pattern (NaN payloads give infinity by design)
        if (i < 0x80000000ULL) {
            const float f = __uint_as_float((unsigned)i);
            const bool nan = f != f;
            const double want = nan ? CUDART_INF : (double)f;
            if (bits(f2d_pos(f)) != __double_as_longlong(want)) atomicAdd(bad + 0, 1ULL);
        }
        const unsigned long long r = mix64(i);
        // f32_trunc: truncation toward zero where the FP32 result is normal or infinite
        const double x = __longlong_as_double((long long)r);
        const int ex = (int)((r >> 52) & 0x7ff) - 1023;
        if (ex >= -126 && x == x) {
            const float want = ex > 127 ? copysignf(CUDART_INF_F, (float)x) : __double2float_rz(x);
            if (__float_as_uint(f32_trunc(x)) != __float_as_uint(want)) atomicAdd(bad + 1, 1ULL);
        }
        // f32_rn_pos: round to nearest even for u >= 2^-126
        const unsigned long long ub = (r & 0x000fffffffffffffULL) | ((unsigned long long)(897 + (r >> 52) % 1150) << 52);
        const double u = __longlong_as_double((long long)ub);
        if (__float_as_uint(f32_rn_pos(u)) != __float_as_uint(__double2float_rn(u))) atomicAdd(bad + 2, 1ULL);
        // frexp_normal on positive normal doubles
        const unsigned long long nb = (r & 0x000fffffffffffffULL) | ((unsigned long long)(1 + (r >> 52) % 2046) << 52);
        int e1, e2;
        const double m1 = frexp_normal(__longlong_as_double((long long)nb), e1);
        const double m2 = frexp(__longlong_as_double((long long)nb), &e2);
        if (bits(m1) != __double_as_longlong(m2) || e1 != e2) atomicAdd(bad + 3, 1ULL);
        // i2d_exact on |e| <= 2^30 and pow2i on [-2000, 2000]
        const int ei = (int)(r % (1ULL << 31)) - (1 << 30);
        if (bits(i2d_exact(ei)) != __double_as_longlong((double)ei)) atomicAdd(bad + 4, 1ULL);
        const int es = (int)(i % 8001) - 4000;
        if (bits(i2d_exact(es)) != __double_as_longlong((double)es)) atomicAdd(bad + 4, 1ULL);
        const int k = (int)(i % 4001) - 2000;
        if (bits(pow2i(k)) != __double_as_longlong(ldexp(1.0, k))) atomicAdd(bad + 5, 1ULL);
    }
}

int main()
{
    unsigned long long* bad = nullptr;
    if (cudaMalloc(&bad, 8 * sizeof(unsigned long long)) != cudaSuccess) return 2;
    cudaMemset(bad, 0, 8 * sizeof(unsigned long long));
    check<<<152 * 8, 256>>>(bad, 0x80000000ULL);
    unsigned long long h[8] = {0};
    cudaMemcpy(h, bad, sizeof h, cudaMemcpyDeviceToHost);
    const cudaError_t e = cudaDeviceSynchronize();
    printf("%s f2d_pos %llu f32_trunc %llu f32_rn_pos %llu frexp %llu i2d %llu pow2i %llu\n", cudaGetErrorString(e),
           h[0], h[1], h[2], h[3], h[4], h[5]);
    cudaFree(bad);
    return (e == cudaSuccess && !(h[0] | h[1] | h[2] | h[3] | h[4] | h[5])) ? 0 : 1;
}
