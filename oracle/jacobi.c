/*
 * Oracle (test infrastructure only; never on the product path).
 *
 * Plain C99 + OpenMP Jacobi sub-solvers for the CPU FP64 oracle of the
 * CS decomposition via two polar decompositions (Algorithm 1).  Instantiated
 * for real (double, suffix _d) and complex (double complex, suffix _z) data.
 * Matrices are column-major with an explicit leading dimension.
 * Built into oracle/liboracle_jacobi.so by oracle/build.py; loaded with ctypes.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>

#ifndef JTOL
#define JTOL 2.0
#endif

#define SCALAR double
#define SUFFIX _d
#define ABS2(x) ((x) * (x))
#define CABS(x) fabs(x)
#define CONJ(x) (x)
#define CREAL(x) (x)
#define CIMAG(x) 0.0
#define IS_COMPLEX 0
#define MAKE(re, im) (re)
#include "jacobi_impl.h"
#undef SCALAR
#undef SUFFIX
#undef ABS2
#undef CABS
#undef CONJ
#undef CREAL
#undef CIMAG
#undef IS_COMPLEX
#undef MAKE

#define SCALAR double complex
#define SUFFIX _z
#define ABS2(x) (creal(x) * creal(x) + cimag(x) * cimag(x))
#define CABS(x) cabs(x)
#define CONJ(x) conj(x)
#define CREAL(x) creal(x)
#define CIMAG(x) cimag(x)
#define IS_COMPLEX 1
#define MAKE(re, im) ((re) + (im) * I)
#include "jacobi_impl.h"
