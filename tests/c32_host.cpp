// Host build of the compensated FP32 element arithmetic (csrc/c32.cuh) for
// the CPU tests: the same source, compiled without contraction, computes
// bitwise what the device computes.
#include "c32.cuh"

using phfem::c32::f2;

extern "C" {

int c32_split(double x, float* hl) {
  f2 o{0.f, 0.f};
  const bool ok = phfem::c32::split(x, o);
  hl[0] = o.h;
  hl[1] = o.l;
  return ok ? 1 : 0;
}

double c32_widen(float x) { return phfem::c32::widen(x); }

float c32_narrow(double x) { return phfem::c32::narrow(x); }

float c32_frcp(float x) { return phfem::c32::frcp(x); }

double c32_to_double(float h, float l) { return phfem::c32::to_double({h, l}); }

void c32_two_sum(float a, float b, float* out) {
  const f2 r = phfem::c32::two_sum(a, b);
  out[0] = r.h;
  out[1] = r.l;
}

// v = (a.h, a.l, b.h, b.l, c.h, c.l, d.h, d.l): a b + c d
void c32_dot2(const float* v, float* out) {
  const f2 r = phfem::c32::dot2({v[0], v[1]}, {v[2], v[3]}, {v[4], v[5]}, {v[6], v[7]});
  out[0] = r.h;
  out[1] = r.l;
}

void c32_rcp(float h, float l, float* out) {
  const f2 r = phfem::c32::rcp({h, l}, phfem::c32::frcp(h));
  out[0] = r.h;
  out[1] = r.l;
}

int c32_tri_record(double x0, double y0, double x1, double y1, double x2, double y2, double a, double* out64) {
  return phfem::c32::tri_record(x0, y0, x1, y1, x2, y2, a, out64) ? 1 : 0;
}

}  // extern "C"
