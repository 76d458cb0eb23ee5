// Code-layout builder: validates a QC base matrix and compiles it into the
// per-layer circulant table the layer kernel reads.
//
// What it encodes comes from arXiv 2004.09084: the base matrix of shifts with
// all-zero blocks (Results, Eq. (m) and the following sentence), the compact
// index file of (shift, row, column) triples with column degrees (Results,
// the H_compact1 paragraph), and the merging of unrelated base rows into one
// layer (Results, Eqs. (m1), (m2)).  The table is our own format: per layer a
// list of rows, per row a list of (variable offset, shift, message slot,
// column) with the row's core columns (degree > 1) first, so that the kernel
// can specialise a row on its (core, degree-1) edge counts.
#include <algorithm>
#include <cstring>

#include "qcmet_internal.h"

namespace qcmet {

namespace {

bool rows_share_column(const Code &c, int32_t a, int32_t b) {
    for (int32_t k = 0; k < c.nb; ++k)
        if (c.base[(size_t)a * c.nb + k] && c.base[(size_t)b * c.nb + k]) return true;
    return false;
}

// Layers as lists of base rows, according to the merge mode.
std::vector<std::vector<int32_t>> make_layers(const Code &c, const std::vector<int32_t> &rows) {
    std::vector<std::vector<int32_t>> layers;
    if (c.merge_mode == QCMET_MERGE_NONE) {
        for (int32_t r : rows) layers.push_back({r});
    } else if (c.merge_mode == QCMET_MERGE_EXACT) {
        // Longest-path layering of the "shares a column and comes earlier"
        // order: every related pair keeps its base order, unrelated rows that
        // are not separated by a related one share a layer.
        std::vector<int32_t> level(c.mb, -1);
        for (size_t i = 0; i < rows.size(); ++i) {
            int32_t lv = 0;
            for (size_t j = 0; j < i; ++j)
                if (rows_share_column(c, rows[j], rows[i])) lv = std::max(lv, level[rows[j]] + 1);
            level[rows[i]] = lv;
            if ((int32_t)layers.size() <= lv) layers.resize(lv + 1);
            layers[lv].push_back(rows[i]);
        }
    } else {
        // First fit: a row joins the first layer whose rows it shares no column with.
        for (int32_t r : rows) {
            bool placed = false;
            for (auto &layer : layers) {
                bool clash = false;
                for (int32_t o : layer)
                    if (rows_share_column(c, o, r)) {
                        clash = true;
                        break;
                    }
                if (!clash) {
                    layer.push_back(r);
                    placed = true;
                    break;
                }
            }
            if (!placed) layers.push_back({r});
        }
    }
    return layers;
}

void pad4(std::vector<int32_t> &w) {
    while (w.size() % 4) w.push_back(0);
}

}  // namespace

int build_code(const int8_t *base, const int32_t *shifts, int32_t mb, int32_t nb, int32_t Z,
               int32_t merge_mode, Code &c, std::string &err) {
    if (!base || !shifts) {
        err = "base and shifts must not be NULL";
        return QCMET_ERR_INVALID_ARG;
    }
    if (mb < 1 || nb < 1 || Z < 1) {
        err = "mb, nb and Z must be >= 1";
        return QCMET_ERR_INVALID_ARG;
    }
    if ((int64_t)nb * Z >= (int64_t)1 << 31 || (int64_t)mb * Z >= (int64_t)1 << 31) {
        err = "n = nb*Z and m = mb*Z must be below 2^31";
        return QCMET_ERR_INVALID_ARG;
    }
    if (merge_mode != QCMET_MERGE_NONE && merge_mode != QCMET_MERGE_EXACT &&
        merge_mode != QCMET_MERGE_GREEDY) {
        err = "unknown merge mode";
        return QCMET_ERR_INVALID_ARG;
    }
    c.mb = mb;
    c.nb = nb;
    c.Z = Z;
    c.merge_mode = merge_mode;
    const size_t cells = (size_t)mb * nb;
    c.base.assign(base, base + cells);
    c.shifts.assign(cells, 0);
    c.col_degree.assign(nb, 0);
    c.circulants = 0;
    c.max_row_degree = 0;
    for (int32_t l = 0; l < mb; ++l) {
        int32_t deg = 0;
        for (int32_t k = 0; k < nb; ++k) {
            const size_t i = (size_t)l * nb + k;
            if (base[i] != 0 && base[i] != 1) {
                err = "base entries must be 0 (zero block) or 1 (circulant); found " +
                      std::to_string((int)base[i]) + " at row " + std::to_string(l) +
                      ", column " + std::to_string(k);
                return QCMET_ERR_INVALID_ARG;
            }
            if (!base[i]) continue;
            if (shifts[i] < 0 || shifts[i] >= Z) {
                err = "shift " + std::to_string(shifts[i]) + " at row " + std::to_string(l) +
                      ", column " + std::to_string(k) + " is outside [0, Z)";
                return QCMET_ERR_SHIFT_RANGE;
            }
            c.shifts[i] = shifts[i];
            ++deg;
            ++c.col_degree[k];
        }
        if (deg > QCMET_MAX_ROW_DEGREE) {
            err = "row " + std::to_string(l) + " has " + std::to_string(deg) +
                  " circulants; the limit is " + std::to_string(QCMET_MAX_ROW_DEGREE);
            return QCMET_ERR_DEGREE_LIMIT;
        }
        c.circulants += deg;
        c.max_row_degree = std::max(c.max_row_degree, deg);
    }

    // rows with circulants are scheduled; rows without any only enter the final syndrome test
    std::vector<int32_t> rows;
    c.zero_rows.clear();
    for (int32_t l = 0; l < mb; ++l) {
        bool any = false;
        for (int32_t k = 0; k < nb && !any; ++k) any = c.base[(size_t)l * nb + k] != 0;
        (any ? rows : c.zero_rows).push_back(l);
    }
    auto layers = make_layers(c, rows);
    c.sched_rows.clear();
    c.layer_first.clear();
    for (auto &layer : layers) {
        c.layer_first.push_back((int32_t)c.sched_rows.size());
        for (int32_t r : layer) c.sched_rows.push_back(r);
    }
    c.layer_first.push_back((int32_t)c.sched_rows.size());

    // message slots: one per circulant on a core column, numbered row-major
    std::vector<int32_t> slot(cells, -1);
    c.msg_slots = 0;
    c.degree1_columns = 0;
    c.core_cols = 0;
    std::vector<int32_t> col_core(nb, -1);
    for (int32_t k = 0; k < nb; ++k) {
        c.degree1_columns += c.col_degree[k] == 1;
        if (c.col_degree[k] > 1) col_core[k] = c.core_cols++;
    }
    for (int32_t l = 0; l < mb; ++l)
        for (int32_t k = 0; k < nb; ++k) {
            const size_t i = (size_t)l * nb + k;
            if (c.base[i] && c.col_degree[k] > 1) slot[i] = c.msg_slots++;
        }

    // flat device image
    ScheduleImage &im = c.image;
    im = ScheduleImage();
    std::vector<int32_t> &w = im.words;
    const int32_t n_layers = (int32_t)layers.size();
    const int32_t n_rows = (int32_t)c.sched_rows.size();
    w.assign(kHdrWords, 0);
    w[kHdrRows] = n_rows;
    w[kHdrLayers] = n_layers;
    w[kHdrEntries] = c.circulants;
    w[kHdrNb] = nb;
    w[kHdrZ] = Z;
    w[kHdrMb] = mb;
    im.off_layer_first = (int32_t)w.size();
    for (int32_t v : c.layer_first) w.push_back(v);
    pad4(w);
    im.off_rows = (int32_t)w.size();
    std::vector<DevEntry> ents;
    for (int32_t r : c.sched_rows) {
        DevRow dr;
        dr.first_entry = (int32_t)ents.size();
        dr.check_base = r * Z;
        dr.row = r;
        // core columns first, then degree-1 columns: the kernel specialises a
        // row on (core edges, degree-1 edges)
        int32_t deg = 0;
        for (int pass = 0; pass < 2; ++pass)
            for (int32_t k = 0; k < nb; ++k) {
                const size_t i = (size_t)r * nb + k;
                if (!c.base[i] || (col_core[k] >= 0) != (pass == 0)) continue;
                const int32_t vb = col_core[k] >= 0 ? col_core[k] * Z : k * Z;
                ents.push_back(DevEntry{vb, c.shifts[i], slot[i], k});
                ++deg;
            }
        dr.degree = deg;
        w.push_back(dr.first_entry);
        w.push_back(dr.degree);
        w.push_back(dr.check_base);
        w.push_back(dr.row);
    }
    im.off_entries = (int32_t)w.size();
    for (const DevEntry &e : ents) {
        w.push_back(e.var_base);
        w.push_back(e.shift);
        w.push_back(e.slot);
        w.push_back(e.col);
    }
    im.off_col_kind = (int32_t)w.size();
    for (int32_t k = 0; k < nb; ++k)
        w.push_back(c.col_degree[k] == 0 ? kColUnconnected
                                         : (c.col_degree[k] == 1 ? kColDegree1 : kColCore));
    pad4(w);
    im.off_zero_rows = (int32_t)w.size();
    im.n_zero_rows = (int32_t)c.zero_rows.size();
    for (int32_t r : c.zero_rows) w.push_back(r);
    pad4(w);
    const int32_t off_col_core = (int32_t)w.size();
    for (int32_t k = 0; k < nb; ++k) w.push_back(col_core[k]);
    pad4(w);
    w[kHdrOffColCore] = off_col_core;
    w[kHdrCoreCols] = c.core_cols;
    w[kHdrMsgSlots] = c.msg_slots;
    w[kHdrOffLayerFirst] = im.off_layer_first;
    w[kHdrOffRows] = im.off_rows;
    w[kHdrOffEntries] = im.off_entries;
    w[kHdrOffColKind] = im.off_col_kind;
    w[kHdrOffZeroRows] = im.off_zero_rows;
    w[kHdrZeroRows] = im.n_zero_rows;
    return QCMET_OK;
}

}  // namespace qcmet
