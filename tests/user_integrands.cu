// Integrands compiled outside the library, as a caller would write them, for
// the user-integrand tests (include/vegas_user_integrand.cuh).
#include "vegas_user_integrand.cuh"

// Eq. 1 in the plain coordinate, parameters from the caller's device data
// [a, mu_1 .. mu_D]: (a sqrt(pi))^-D exp(-sum_k (x_k - mu_k)^2 / a^2), the
// same function as the built-in VEGAS_GAUSS, evaluated another way.
struct UserGauss {
    template <typename R, int D>
    __device__ R operator()(const R (&x)[D], const void* data) const {
        const double* p = static_cast<const double*>(data);
        const R inv_a = (R)(1.0 / p[0]);
        R s = 0;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const R z = (x[k] - (R)p[1 + k]) * inv_a;
            s += z * z;
        }
        const R norm = (R)pow(p[0] * 1.7724538509055160273, -(double)D);
        return norm * exp(-s);
    }
};

// (x_1 + ... + x_D)^2: not a product over dimensions; its integral over the
// unit cube is D/12 + D^2/4.
struct UserSumSquare {
    template <typename R, int D>
    __device__ R operator()(const R (&x)[D], const void*) const {
        R s = 0;
#pragma unroll
        for (int k = 0; k < D; ++k) s += x[k];
        return s * s;
    }
};

// prod_k (pi/2) sin(pi x_k): integral 1, zero on the faces of the cube.
struct UserSine {
    template <typename R, int D>
    __device__ R operator()(const R (&x)[D], const void*) const {
        R f = 1;
#pragma unroll
        for (int k = 0; k < D; ++k) f *= (R)1.5707963267948966 * sin((R)3.141592653589793 * x[k]);
        return f;
    }
};

// NaN where x_1 < 1/4, else 1: on a uniform grid of 4 bins the non-finite
// samples are exactly those in the first bin of dimension 1.
struct UserHole {
    template <typename R, int D>
    __device__ R operator()(const R (&x)[D], const void*) const {
        return x[0] < (R)0.25 ? (R)NAN : (R)1;
    }
};

VEGAS_USER_INTEGRAND(user_gauss_d4, UserGauss, 4)
VEGAS_USER_INTEGRAND(user_hole_d2, UserHole, 2)
VEGAS_USER_INTEGRAND(user_gauss_d8, UserGauss, 8)
VEGAS_USER_INTEGRAND(user_sum_square_d5, UserSumSquare, 5)
VEGAS_USER_INTEGRAND(user_sine_d3, UserSine, 3)
