// Forward-mode dual numbers for the gradient kernel: a value and its
// derivatives with respect to NT parameters.  The intersection and
// interaction templates of trace.cuh are instantiated with this type to
// carry derivatives along a photon's frozen path; every branch decides on
// the value, so the path is the one the plain trace takes.
#pragma once
#include "trace.cuh"

namespace robast {

template <typename R, int NT>
struct Dn {
    R v;
    R d[NT];
    __device__ __forceinline__ Dn() {}
    __device__ __forceinline__ Dn(double x) : v((R)x) {
#pragma unroll
        for (int k = 0; k < NT; ++k) d[k] = R(0);
    }
    __device__ __forceinline__ Dn(float x) : v((R)x) {
#pragma unroll
        for (int k = 0; k < NT; ++k) d[k] = R(0);
    }
    __device__ __forceinline__ Dn(int x) : v((R)x) {
#pragma unroll
        for (int k = 0; k < NT; ++k) d[k] = R(0);
    }
    friend __device__ __forceinline__ Dn operator+(const Dn& a, const Dn& b) {
        Dn r;
        r.v = a.v + b.v;
#pragma unroll
        for (int k = 0; k < NT; ++k) r.d[k] = a.d[k] + b.d[k];
        return r;
    }
    friend __device__ __forceinline__ Dn operator-(const Dn& a, const Dn& b) {
        Dn r;
        r.v = a.v - b.v;
#pragma unroll
        for (int k = 0; k < NT; ++k) r.d[k] = a.d[k] - b.d[k];
        return r;
    }
    friend __device__ __forceinline__ Dn operator-(const Dn& a) {
        Dn r;
        r.v = -a.v;
#pragma unroll
        for (int k = 0; k < NT; ++k) r.d[k] = -a.d[k];
        return r;
    }
    friend __device__ __forceinline__ Dn operator*(const Dn& a, const Dn& b) {
        Dn r;
        r.v = a.v * b.v;
#pragma unroll
        for (int k = 0; k < NT; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
        return r;
    }
    friend __device__ __forceinline__ Dn operator/(const Dn& a, const Dn& b) {
        Dn r;
        r.v = a.v / b.v;
        const R ib = R(1) / b.v;
#pragma unroll
        for (int k = 0; k < NT; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) * ib;
        return r;
    }
    __device__ __forceinline__ Dn& operator+=(const Dn& b) { return *this = *this + b; }
    __device__ __forceinline__ Dn& operator-=(const Dn& b) { return *this = *this - b; }
    __device__ __forceinline__ Dn& operator*=(const Dn& b) { return *this = *this * b; }
    friend __device__ __forceinline__ bool operator<(const Dn& a, const Dn& b) { return a.v < b.v; }
    friend __device__ __forceinline__ bool operator<=(const Dn& a, const Dn& b) { return a.v <= b.v; }
    friend __device__ __forceinline__ bool operator>(const Dn& a, const Dn& b) { return a.v > b.v; }
    friend __device__ __forceinline__ bool operator>=(const Dn& a, const Dn& b) { return a.v >= b.v; }
    friend __device__ __forceinline__ bool operator==(const Dn& a, const Dn& b) { return a.v == b.v; }
    friend __device__ __forceinline__ bool operator!=(const Dn& a, const Dn& b) { return a.v != b.v; }
};

template <typename R, int NT>
__device__ __forceinline__ Dn<R, NT> t_sqrt(const Dn<R, NT>& x) {
    Dn<R, NT> r;
    r.v = t_sqrt(x.v);
    const R h = R(0.5) / r.v;
#pragma unroll
    for (int k = 0; k < NT; ++k) r.d[k] = x.d[k] * h;
    return r;
}
template <typename R, int NT>
__device__ __forceinline__ Dn<R, NT> t_abs(const Dn<R, NT>& x) {
    return x.v >= R(0) ? x : -x;
}
template <typename R, int NT>
__device__ __forceinline__ Dn<R, NT> t_min(const Dn<R, NT>& a, const Dn<R, NT>& b) {
    return b.v < a.v ? b : a;
}
template <typename R, int NT>
__device__ __forceinline__ Dn<R, NT> t_max(const Dn<R, NT>& a, const Dn<R, NT>& b) {
    return b.v > a.v ? b : a;
}

template <typename T>
__device__ __forceinline__ T t_inf_of();
template <>
__device__ __forceinline__ float t_inf_of<float>() { return t_inf<float>(); }
template <>
__device__ __forceinline__ double t_inf_of<double>() { return t_inf<double>(); }

}  // namespace robast
