/*
 * tpc_reduce.h -- data-reduction calls of libtpc.so (arXiv:1910.12214, Sec. 4,
 * "TPC Data Reduction").  They share the context, status codes and conventions
 * of tpc.h: every call returns a tpc_status and never aborts; device work runs
 * on the context's stream.
 */
#ifndef TPC_REDUCE_H
#define TPC_REDUCE_H

#include "tpc.h"

#ifdef __cplusplus
extern "C" {
#endif

/* ---- Cluster codec (Sec. 4, step 2) -------------------------------------
 *
 * Converts cluster properties from the reconstruction's floating-point format
 * to integers carrying only the precision the detector resolves.  The paper
 * fixes the dynamic precision of cluster size and charge: in the integer
 * representation every bit more than n places after the leading one is
 * cleared, with rounding, n = 3 for sizes and n = 4 for charges.  Field units
 * and widths are this library's choice (the paper gives none):
 *
 *   field     input        code                      step
 *   y         float  [cm]  int16, nearest (ties even) 2^-6 cm, saturated
 *   z         float  [cm]  int32, nearest (ties even) 2^-6 cm, saturated
 *   row       int32        uint8                      pad row; 0 if out of range
 *   q_tot     float [ADC]  uint16, nearest (ties even) 1 ADC count, saturated,
 *   q_max     float [ADC]  uint16                      then n = 4 dynamic precision
 *   sigma_y   float  [cm]  uint8, nearest (ties even) 2^-7 cm, saturated,
 *   sigma_z   float  [cm]  uint8                      then n = 3 dynamic precision
 *
 * Dynamic precision rounds to the nearest value with n bits after its leading
 * one (ties upward); a carry out of the field gives the largest such value
 * that fits (0xF800 for charges, 0xF0 for sizes).  Negative charges and sizes
 * code as 0; NaN codes as 0 in every field.
 *
 * The decoded value of a code is code x step. */
#define TPC_CODE_POS_STEP_CM (1.0 / 64.0)
#define TPC_CODE_SIZE_STEP_CM (1.0 / 128.0)
#define TPC_CODE_CHARGE_BITS 4 /* bits kept after the leading one */
#define TPC_CODE_SIZE_BITS 3

/* n clusters in SoA form.  Arrays of n values each, all host or all device
 * pointers (see on_device below). */
typedef struct {
  const float* y;
  const float* z;
  const int32_t* row;
  const float* q_tot;
  const float* q_max;
  const float* sigma_y;
  const float* sigma_z;
  uint64_t n;
} tpc_cluster_props;

/* Output codes, n values per array, owned by the caller. */
typedef struct {
  int16_t* y;
  int32_t* z;
  uint8_t* row;
  uint16_t* q_tot;
  uint16_t* q_max;
  uint8_t* sigma_y;
  uint8_t* sigma_z;
} tpc_cluster_codes;

/* Encodes in->n clusters into *out.
 *  on_device = 0: every pointer is a host pointer; the call copies the
 *    properties to the device (staging buffers kept by the context), encodes,
 *    copies the codes back and waits.
 *  on_device = 1: every pointer is a device pointer on the context's device;
 *    the work is enqueued on the context's stream.  With n_bad == NULL the call
 *    returns at once and bad clusters are coded but not reported; otherwise it
 *    waits for the stream.
 * A cluster is bad if its row is outside [0, n_rows) of the context or a value
 * is not finite; it is coded by the rules above all the same.  *n_bad
 * (nullable) receives their number and the call returns TPC_ERR_BAD_INPUT when
 * it is not zero.  n = 0 is valid (nothing happens).  A NULL array with n > 0
 * gives TPC_ERR_INVALID_ARG.  Device arrays aligned to 16 bytes (inputs, z)
 * and 8 bytes (y, charges) take a vectorised path; other alignments are valid
 * and slower. */
tpc_status tpc_encode_clusters(tpc_ctx* ctx, const tpc_cluster_props* in, const tpc_cluster_codes* out, int on_device,
                               uint64_t* n_bad);

#ifdef __cplusplus
}
#endif
#endif /* TPC_REDUCE_H */
