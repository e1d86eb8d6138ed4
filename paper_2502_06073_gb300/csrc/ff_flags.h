/*
 * Device error word of libff: the bits that kernels set with atomicOr in a word the host
 * reads back after the launches that can fail, and the one mapping from that word to the
 * ABI's status codes.  Plain C (no CUDA headers) so the mapping can be compiled and
 * checked on a host without a GPU.
 */
#ifndef FF_FLAGS_H_
#define FF_FLAGS_H_

#include "../../include/ff.h"

#define FF_FLAG_CAPACITY 1        /* a neighbour count exceeded the list capacity */
#define FF_FLAG_BOX 4             /* an image shift beyond 100 box lengths */
#define FF_FLAG_REVERSE 8         /* an edge without its reverse (asymmetric list) */
#define FF_FLAG_SPECIES 16        /* an atomic number outside 1..89 */
#define FF_FLAG_NONFINITE_F 32    /* a non-finite force */
#define FF_FLAG_TIMEOUT 64        /* a bounded device wait (tensor-core pipeline) ran out */
#define FF_FLAG_NONFINITE_POS 128 /* a non-finite position */

/* Status of an error word (FF_OK for 0).  When several bits are set the first in the order
 * below wins: a bad input (species, position, box) is reported before what it causes.
 * *what (may be NULL) receives a static description. */
static inline int ff_flags_status(int word, const char** what) {
  const char* w = "";
  int st = FF_OK;
  if (word & FF_FLAG_SPECIES) {
    w = "atomic number outside 1..89";
    st = FF_ERR_SPECIES;
  } else if (word & FF_FLAG_NONFINITE_POS) {
    w = "non-finite position";
    st = FF_ERR_NONFINITE;
  } else if (word & FF_FLAG_BOX) {
    w = "periodic image shift beyond 100 box lengths";
    st = FF_ERR_BOX;
  } else if (word & FF_FLAG_CAPACITY) {
    w = "neighbour count above the per-atom limit";
    st = FF_ERR_CAPACITY;
  } else if (word & FF_FLAG_REVERSE) {
    w = "reverse edge missing (asymmetric list)";
    st = FF_ERR_STATE;
  } else if (word & FF_FLAG_TIMEOUT) {
    w = "tensor-core GEMM pipeline wait timed out (outputs of that evaluation are invalid)";
    st = FF_ERR_TIMEOUT;
  } else if (word & FF_FLAG_NONFINITE_F) {
    w = "non-finite force";
    st = FF_ERR_NONFINITE;
  } else if (word) {
    w = "unknown device error bit";
    st = FF_ERR_CUDA;
  }
  if (what) *what = w;
  return st;
}

#endif /* FF_FLAGS_H_ */
