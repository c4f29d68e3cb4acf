// export.cu -- headless image export: the rendered colour and id planes packed
// into interleaved 8-bit RGBA with a background of chosen transparency (the
// alpha of pixels where no primitive was hit), ready to be written to an
// image file by the host.
#include "vtx_internal.h"

namespace vtx {

// One pixel per thread and grid-stride iteration: three colour planes and the
// id plane read coalesced, one 32-bit RGBA word written.  HBM-bound
// (16 B read + 4 B written per pixel).
__global__ __launch_bounds__(256) void k_export_rgba8(const float *__restrict__ rgb, const uint32_t *__restrict__ id,
                                                      long long ppi, long long n_px, unsigned char bg_a,
                                                      uchar4 *__restrict__ out) {
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n_px;
       q += (long long)gridDim.x * blockDim.x) {
    const long long img = q / ppi, p = q - img * ppi;
    const float *c = rgb + img * 3 * ppi + p;
    uchar4 o;
    o.x = (unsigned char)__float2uint_rn(fminf(fmaxf(__ldcs(c), 0.0f), 1.0f) * 255.0f);
    o.y = (unsigned char)__float2uint_rn(fminf(fmaxf(__ldcs(c + ppi), 0.0f), 1.0f) * 255.0f);
    o.z = (unsigned char)__float2uint_rn(fminf(fmaxf(__ldcs(c + 2 * ppi), 0.0f), 1.0f) * 255.0f);
    o.w = __ldcs(id + q) == kNoId ? bg_a : 255;
    __stcs(out + q, o);
  }
}

cudaError_t run_export_rgba8(const float *rgb, const uint32_t *id, long long ppi, long long n_img, unsigned char bg_a,
                             uint8_t *rgba, cudaStream_t st) {
  const long long n = ppi * n_img;
  if (n == 0) return cudaSuccess;
  const long long blocks = (n + 255) / 256;
  const long long cap = 8LL * sm_count();
  k_export_rgba8<<<(int)(blocks < cap ? blocks : cap), 256, 0, st>>>(rgb, id, ppi, n, bg_a,
                                                                     reinterpret_cast<uchar4 *>(rgba));
  return cudaGetLastError();
}

}  // namespace vtx
