// Record stream of the batched local solves (host builder: snode_plan.cpp; consumer:
// k_sn_stream in kernels_snode.cu).  Plain structs, usable from host and device code.
//
// Every warp of a solve CTA owns one byte stream per subdomain: the records of the work
// units it is given, in the order it processes them, each record 16-byte aligned and
// holding a 16-byte header (SnRec), an optional index list and its factor entries.  The
// warp copies its stream into a private shared-memory ring with bulk async copies ahead
// of use and interprets it record by record; nothing else is read from global memory.
//
// A unit is a supernode J of the subdomain and a chunk of up to 32 of its rows
// (forward: lane = row) or columns (backward: lane = column); t0 = its first row.  Entries
// are stored in groups of V = 8 / sizeof(entry) along the loop direction, so that a lane
// reads a group with one 8-byte load and consecutive lanes read consecutive groups;
// groups are padded with zeros (and padding rows of SN_BPANEL carry index 0).
//   SN_FCONTRIB  forward: `rows` consecutive panel rows of a descendant K, columns
//                [x0 - c0_K, + ncols) of K, preceded by `rows` uint8 target lanes (padded
//                to 16 bytes); entry (i, c) at (c / V) rows V + i V + c % V.
//                acc[target(i)] -= row_i . y[x0 ..]
//                (FIRST: acc = v[t0 + lane]; LAST: v[t0 + lane] = acc)
//   SN_FDIAG     forward: columns [x0 - c0_J, + ncols) of D_J for the unit's rows; column
//                group g (columns x0 + gV ..) holds the rows l >= st(g) = max(0, rel0 + gV),
//                rel0 = x0 - t0; entry (l, c) at sn_fdiag_off(g) + (l - st(g)) V + (c - x0) % V.
//                yacc += D[., c] v[c]  (FIRST: yacc = 0; LAST: y[t0 + lane] = yacc)
//   SN_BPANEL    backward: `rows` rows of L_{R_J,J} restricted to the unit's columns,
//                preceded by the rows' subdomain-local indices (uint16, one group of V per
//                V rows, padded to 16 bytes); entry (i, c) at (i / V) lanes V + c V + i % V.
//                acc -= column . v[R]  (FIRST: acc = y[t0 + lane]; LAST: y[t0 + lane] = acc)
//   SN_BDIAG     backward: rows [x0 - c0_J, + ncols) of D_J restricted to the unit's
//                columns; row group g (rows x0 + gV ..) holds the columns
//                c < min(lanes, rel0 + gV + V), rel0 = x0 - t0 >= 0; entry (r, c) at
//                sn_bdiag_off(g) + c V + (r - x0) % V.
//                xacc += D[r, .] y[r]  (FIRST: xacc = 0; LAST: v[t0 + lane] = xacc)
//   SN_BARRIER   CTA barrier; every warp's stream of a subdomain holds the same number.
//   SN_END       end of the stream.
#pragma once

#include <cstdint>

namespace am {

enum : uint8_t { SN_END = 0, SN_BARRIER = 1, SN_FCONTRIB = 2, SN_FDIAG = 3, SN_BPANEL = 4, SN_BDIAG = 5 };
enum : uint8_t { SN_FIRST = 1, SN_LAST = 2 };

struct SnRec {
    uint8_t kind, flags;
    uint8_t lanes;      // lanes of the unit (rows forward, columns backward), <= 32
    uint8_t rows;       // FCONTRIB: block rows; BPANEL: panel rows in this record
    uint16_t t0;        // first row of the unit (subdomain-local)
    uint16_t x0;        // FCONTRIB: y index of the first column; FDIAG: v index of the first column;
                        // BDIAG: y index of the first row
    uint16_t ncols;     // FCONTRIB / FDIAG: columns in the record; BDIAG: rows in the record
    uint16_t hdr;       // bytes between the header and the entries (index list)
    uint32_t bytes;     // record size, header included, multiple of 16
};
static_assert(sizeof(SnRec) == 16, "16-byte record header");

// Where the finalisation kernel takes a record's entries from (the factor fronts and
// the row-major packed inverse diagonal blocks of the numeric factorisation).
struct SnFill {
    int64_t off;        // byte offset of the record's entries in the stream
    int32_t sn;         // source supernode (global index): K for FCONTRIB, J otherwise
    uint8_t kind, lanes, rows, pad;
    uint16_t p0;        // FCONTRIB: first panel row of K; FDIAG: unit's first row (J-local);
                        // BPANEL: first panel row; BDIAG: unit's first column (J-local)
    uint16_t p1;        // FCONTRIB: first column of K; FDIAG: first column; BPANEL: unit's first
                        // column (J-local); BDIAG: first row
    uint16_t n;         // FCONTRIB / FDIAG: columns; BPANEL / BDIAG: rows
    uint16_t pad2;
};
static_assert(sizeof(SnFill) == 24, "fill descriptor");

#ifdef __CUDACC__
#define SN_HD __host__ __device__ __forceinline__
#else
#define SN_HD inline
#endif

// Entries before group g of an SN_FDIAG record (lanes L, rel0 = x0 - t0, V per group):
// V sum_{g' < g} (L - max(0, rel0 + g' V)).
SN_HD int64_t sn_fdiag_off(int g, int rel0, int L, int V) {
    const int nz = rel0 >= 0 ? 0 : (g < (-rel0) / V + 1 ? g : (-rel0) / V + 1);
    const int64_t rest = g - nz;
    return (int64_t)V * ((int64_t)nz * L + rest * (L - rel0) - (int64_t)V * (rest * (2 * nz + rest - 1) / 2));
}
// Entries before group g of an SN_BDIAG record (rel0 >= 0): V sum_{g' < g} min(L, rel0 + (g' + 1) V).
SN_HD int64_t sn_bdiag_off(int g, int rel0, int L, int V) {
    int nt = L - rel0 - 1 >= 0 ? (L - rel0 - 1) / V : 0;
    nt = nt < g ? nt : g;
    return (int64_t)V * ((int64_t)nt * rel0 + (int64_t)V * nt * (nt + 1) / 2 + (int64_t)(g - nt) * L);
}

}  // namespace am
