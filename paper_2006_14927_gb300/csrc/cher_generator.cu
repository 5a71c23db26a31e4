// cher_generator.cu -- shower steps from a parameterised electromagnetic
// shower, generated on the device (an extension: the paper's input are the
// EGS4 electron/positron steps that CORSIKA hands to CERENK; this stands in
// for them so that a batch of showers needs no step arrays from the host).
//
// Per shower: primary energy E0, axis (zenith, azimuth), core at h_obs and a
// step count; per step g (global index), eight deviates from
// Philox4x32-10 keyed by the seed, counters (g, 0, 1) and (g, 1, 1):
//   u0: depth t (radiation lengths) from the Greisen profile
//       N(t) ~ exp(t (1 - 1.5 ln s)), s = 3t/(t + 2y), y = ln(E0/85 MeV), on
//       (0, t_g] (t_g: slant depth of h_obs in isothermal air,
//       X = 1030 exp(-h / 8000 m) g/cm^2, X0 = 36.7 g/cm^2), by inverting
//       its CDF tabulated on uniform nodes, linearly between them;
//       height h = 8000 ln(1030 / (t X0 cos zenith)), at most 29999 m;
//   u1, u2: lateral offset -50 ln(u1) m at azimuth 2 pi u2 around the axis;
//   u3: kinetic energy 20 MeV * 250^u3;
//   u4, u5: Box-Muller normals n1, n2; direction axis + sigma (n1 b1 + n2 b2)
//       normalised, sigma = 3 deg * 50 MeV / E;
//   u6: length 1 + 19 u6 m; start time (s_ref - s) / c, s the distance up
//       the axis, s_ref = (30000 m - h_obs) / cos zenith.
// The per-step arithmetic is FP32 (the steps feed the FP32 path; positions
// to ~1e-6 relative); the CDF tables are integrated in FP64 on the host
// (greisen_cdf_host in cher_tables.cpp).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "cher_device.cuh"
#include "cher_internal.h"

namespace cher {

namespace {

// a uniform deviate in (0, 1] with the full relative precision of a float
// near 0 (its logarithm is taken)
__device__ __forceinline__ float u01_full(uint32_t x) {
    return __uint2float_rn(x) * 2.3283064365386963e-10f + 1.1641532182693481e-10f;
}

__global__ void k_generate_steps(const GenParams g) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < g.n;
         i += int64_t(gridDim.x) * blockDim.x) {
        // the shower of step i: the last first-index <= i
        int lo = 0, hi = g.n_showers;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(g.first + mid) <= i) lo = mid; else hi = mid;
        }
        const GenShower S = g.showers[lo];
        const uint32_t c0 = static_cast<uint32_t>(i), c1 = static_cast<uint32_t>(i >> 32);
        const uint4 w0 = dev::philox4x32_10(make_uint4(c0, c1, 0u, 1u), g.key0, g.key1);
        const uint4 w1 = dev::philox4x32_10(make_uint4(c0, c1, 1u, 1u), g.key0, g.key1);
        // depth from the tabulated CDF of this shower
        const float *F = g.cdf + static_cast<int64_t>(lo) * g.n_cdf;
        const float u0 = u01_full(w0.x);
        int a = 0, b = g.n_cdf - 1;
        while (b - a > 1) {
            const int mid = (a + b) >> 1;
            if (__ldg(F + mid) <= u0) a = mid; else b = mid;
        }
        const float Fa = __ldg(F + a), Fb = __ldg(F + a + 1);
        const float frac = Fb > Fa ? fminf(fmaxf((u0 - Fa) / (Fb - Fa), 0.0f), 1.0f) : 0.0f;
        const float t = (static_cast<float>(a) + frac) * S.dt;
        float h = 8000.0f * logf(1030.0f / (t * S.x0cz));
        h = fminf(h, 29999.0f);
        const float sa = (h - g.h_obs) / S.cz;
        const float r = -50.0f * logf(u01_full(w0.y));
        float sp, cp;
        sincospif(2.0f * u01_full(w0.z), &sp, &cp);
        const float lx = r * cp, ly = r * sp;
        g.x0[i] = S.core_x - sa * S.ax + lx * S.b1x + ly * S.b2x;
        g.y0[i] = S.core_y - sa * S.ay + lx * S.b1y + ly * S.b2y;
        g.z0[i] = g.h_obs - sa * S.az + lx * S.b1z + ly * S.b2z;
        const float e = 20.0f * expf(u01_full(w0.w) * 5.52146091786225f);   // ln 250
        g.ekin[i] = e;
        const float sig = 0.05235987755982988f * (50.0f / e);                 // 3 deg
        const float rho = sqrtf(-2.0f * logf(u01_full(w1.x)));
        float s5, c5;
        sincospif(2.0f * u01_full(w1.y), &s5, &c5);
        const float n1 = rho * c5, n2 = rho * s5;
        const float dx = S.ax + sig * (n1 * S.b1x + n2 * S.b2x);
        const float dy = S.ay + sig * (n1 * S.b1y + n2 * S.b2y);
        const float dz = S.az + sig * (n1 * S.b1z + n2 * S.b2z);
        const float inv = 1.0f / sqrtf(dx * dx + dy * dy + dz * dz);
        if (g.dirs_fp32) {
            static_cast<float *>(g.ux)[i] = dx * inv;
            static_cast<float *>(g.uy)[i] = dy * inv;
            static_cast<float *>(g.uz)[i] = dz * inv;
        } else {
            static_cast<double *>(g.ux)[i] = dx * inv;
            static_cast<double *>(g.uy)[i] = dy * inv;
            static_cast<double *>(g.uz)[i] = dz * inv;
        }
        g.t0[i] = (S.s_ref - sa) * 3.3356409519815204f;                      // 1 / c, ns/m
        g.len[i] = 1.0f + 19.0f * u01_full(w1.z);
        g.shower[i] = static_cast<uint32_t>(lo);
    }
}

}  // namespace

cudaError_t generate_steps(const GenParams &g, int num_sms, void *stream) {
    if (g.n <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((g.n + 255) / 256, int64_t(num_sms) * 16);
    k_generate_steps<<<static_cast<int>(blocks), 256, 0, static_cast<cudaStream_t>(stream)>>>(g);
    return cudaGetLastError();
}

}  // namespace cher
