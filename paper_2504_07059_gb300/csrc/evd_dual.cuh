// evd_dual.cuh -- forward-mode dual numbers for the adjoint of the collision.
//
// Dual<N> carries a value and N directional derivatives.  The node-local
// collision (moments, tau_ij, equilibria, cross collision, forcing) is
// written once as templates over its arithmetic type; instantiated with
// Dual<N>, with the N tangents seeded on the node's populations and on the
// parameters, it yields the exact Jacobian of f* at the node, from which the
// adjoint takes its transpose-vector product.  Only the operations those
// templates use are provided.  Loops over the tangents unroll for up to 8
// tangents (registers) and stay rolled above (the tangents then live in local
// memory, which keeps compile times reasonable).
#pragma once

#include <cmath>

namespace evd {

template <int N>
struct Dual {
    double v;
    double d[N];

    Dual() = default;   // trivial (shared-memory tables); Dual(0.0) for a zero
    __host__ __device__ Dual(double x) : v(x)
    {
#pragma unroll (N <= 8 ? N : 1)
        for (int k = 0; k < N; ++k) d[k] = 0.0;
    }
    __host__ __device__ explicit operator double() const { return v; }

    __host__ __device__ Dual& operator+=(const Dual& b)
    {
        v += b.v;
#pragma unroll (N <= 8 ? N : 1)
        for (int k = 0; k < N; ++k) d[k] += b.d[k];
        return *this;
    }
    __host__ __device__ Dual& operator-=(const Dual& b)
    {
        v -= b.v;
#pragma unroll (N <= 8 ? N : 1)
        for (int k = 0; k < N; ++k) d[k] -= b.d[k];
        return *this;
    }
    __host__ __device__ Dual& operator*=(const Dual& b)
    {
#pragma unroll (N <= 8 ? N : 1)
        for (int k = 0; k < N; ++k) d[k] = d[k] * b.v + v * b.d[k];
        v *= b.v;
        return *this;
    }
};

template <int N>
__host__ __device__ inline Dual<N> operator+(Dual<N> a, const Dual<N>& b) { return a += b; }
template <int N>
__host__ __device__ inline Dual<N> operator-(Dual<N> a, const Dual<N>& b) { return a -= b; }
template <int N>
__host__ __device__ inline Dual<N> operator*(Dual<N> a, const Dual<N>& b) { return a *= b; }
template <int N>
__host__ __device__ inline Dual<N> operator-(const Dual<N>& a)
{
    Dual<N> r;
    r.v = -a.v;
    
#pragma unroll (N <= 8 ? N : 1)
        for (int k = 0; k < N; ++k) r.d[k] = -a.d[k];
    return r;
}
// (a/b)' = (a' - (a/b) b') / b
template <int N>
__host__ __device__ inline Dual<N> operator/(const Dual<N>& a, const Dual<N>& b)
{
    Dual<N> r;
    r.v = a.v / b.v;
    const double ib = 1.0 / b.v;
    
#pragma unroll (N <= 8 ? N : 1)
        for (int k = 0; k < N; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) * ib;
    return r;
}
template <int N>
__host__ __device__ inline Dual<N> fma(const Dual<N>& a, const Dual<N>& b, const Dual<N>& c)
{
    Dual<N> r;
    r.v = a.v * b.v + c.v;
    
#pragma unroll (N <= 8 ? N : 1)
        for (int k = 0; k < N; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k] + c.d[k];
    return r;
}
template <int N>
__host__ __device__ inline bool operator>(const Dual<N>& a, const Dual<N>& b) { return a.v > b.v; }
template <int N>
__host__ __device__ inline bool operator<(const Dual<N>& a, const Dual<N>& b) { return a.v < b.v; }
template <int N>
__host__ __device__ inline bool operator!=(const Dual<N>& a, const Dual<N>& b) { return a.v != b.v; }
template <int N>
__host__ __device__ inline bool isfinite(const Dual<N>& a) { return ::isfinite(a.v); }

}  // namespace evd
