"""Planted mistakes: each test replaces one oracle step by a plausible wrong version (on the CPU)
and checks that the pins of test_oracle_pins.py catch it. This shows the pins constrain every
step of the oracle, not only its self-consistency."""
import os

import numpy as np
import pytest

import tests.test_oracle_pins as P
from oracle import numarck_oracle as O

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

PINS = [
    lambda: P.test_grid_constants_dyadic(np.float64),
    lambda: P.test_grid_constants_dyadic(np.float32),
    P.test_change_ratio_closed_forms,
    lambda: P.test_bin_ids_dyadic_centres_and_edges(np.float64),
    P.test_bin_ids_monotone_in_ratio,
    P.test_min_anchor_puts_minimum_in_bin_zero,
    P.test_min_anchor_zero_minimum_is_positive_zero,
    P.test_histogram_hand_counted,
    P.test_top_k_matches_brute_force,
    P.test_top_k_fewer_bins_than_k_selects_all,
    P.test_dp_optimum_reached_on_grid_aligned_clusters,
    lambda: P.test_centres_closed_form(np.float64),
    lambda: P.test_worked_example(GOLDEN),
    P.test_value_space_check_rejects_decreasing_edge_point,
    P.test_unchanged_points_reconstruct_exactly_zero_anchor,
    P.test_error_bound_holds_exactly_for_compressible_points,
    P.test_special_inputs_become_markers_and_roundtrip_bits,
    P.test_pack_hand_example,
    lambda: P.test_pack_matches_integer_bit_writer_and_roundtrips(5),
    lambda: P.test_fig2_block_layout(GOLDEN),
    P.test_offsets_tables_are_prefix_counts,
    P.test_decompress_closed_form,
    P.test_decompress_range_equals_slice,
    P.test_file_size_hand_example,
    P.test_choose_B_single_bin_and_uniform_bins,
    P.test_choose_B_tie_goes_to_smaller_B,
]


def _some_pin_fails() -> bool:
    for pin in PINS:
        try:
            with np.errstate(all="ignore"):
                pin()
        except Exception:
            return True
    return False


def test_pins_pass_on_the_unmodified_oracle():
    assert not _some_pin_fails()


def _ratio_over_cur(prev, cur, cap):
    with np.errstate(all="ignore"):
        r = (cur - prev) / cur
    return r, np.isfinite(r) & (np.abs(r) <= cap)


def _ratio_wrong_sign(prev, cur, cap):
    with np.errstate(all="ignore"):
        r = (prev - cur) / prev
    return r, np.isfinite(r) & (np.abs(r) <= cap)


def _bins_round(ratio, binnable, a, inv_w):
    with np.errstate(all="ignore"):
        u = (ratio - a) * inv_w
    b = np.zeros(ratio.shape, dtype=np.int64)
    b[binnable] = np.round(u[binnable]).astype(np.int64)
    return b


def _bins_anchor_sign(ratio, binnable, a, inv_w):
    with np.errstate(all="ignore"):
        u = (ratio + a) * inv_w
    b = np.zeros(ratio.shape, dtype=np.int64)
    b[binnable] = np.floor(u[binnable]).astype(np.int64)
    return b


def _anchor_keeps_signed_zero(ratio, binnable, E_T, anchor):
    T = type(E_T)
    if anchor == O.ANCHOR_ZERO:
        return T(-E_T)
    return T(ratio[binnable].min()) if binnable.any() else T(0)


def _topk_ties_to_larger(bins, counts, k):
    order = np.lexsort((-bins, -counts))
    return np.sort(bins[order[:k]])


def _topk_count_order(bins, counts, k):
    order = np.lexsort((bins, -counts))
    return bins[order[:k]]


def _centres_no_half(selected, a, w, T):
    return (a + (selected.astype(T) * w)).astype(T)


def _assign_no_check(prev, cur, binnable, b, selected, centres, E_T, M):
    idx = np.full(prev.shape[0], M, dtype=np.int64)
    if selected.size == 0:
        return idx
    pos = np.minimum(np.searchsorted(selected, b), selected.size - 1)
    take = binnable & (selected[pos] == b)
    idx[take] = pos[take]
    return idx


def _assign_prev_tol(prev, cur, binnable, b, selected, centres, E_T, M):
    T = type(E_T)
    idx = np.full(prev.shape[0], M, dtype=np.int64)
    if selected.size == 0:
        return idx
    pos = np.minimum(np.searchsorted(selected, b), selected.size - 1)
    in_sel = binnable & (selected[pos] == b)
    m = (T(1) + centres).astype(T)
    with np.errstate(all="ignore"):
        ok = np.abs(prev * m[pos] - cur) <= E_T * np.abs(prev)
    take = in_sel & ok
    idx[take] = pos[take]
    return idx


def _pack_msb_first(indices, B):
    if indices.size == 0:
        return b""
    bits = ((indices[:, None] >> np.arange(B - 1, -1, -1)[None, :]) & 1).astype(np.uint8)
    return np.packbits(bits.reshape(-1), bitorder="little").tobytes()


def _epb_plus_one(block_bytes, B):
    return (8 * block_bytes) // B + 1


def _grid_width_E(T, E):
    E_T = T(E)
    w = E_T
    inv_w = T(T(1) / w)
    return E_T, w, inv_w, T(w * T(2 ** 21))


def _hist_counts_all(b, binnable):
    bins, counts = np.unique(b, return_counts=True)
    return bins.astype(np.int64), counts.astype(np.int64)


def _sizes_k_is_2_pow_B(counts, n, L, B_max=16):
    desc = np.sort(np.asarray(counts, dtype=np.int64))[::-1]
    prefix = np.concatenate([[0], np.cumsum(desc, dtype=np.int64)])
    return [8 * (1 << B) * L + n * B + 8 * L * (n - int(prefix[min(1 << B, desc.size)]))
            for B in range(1, B_max + 1)]


def _choose_B_ties_to_larger(counts, n, L, B_max=16):
    bits = O.file_size_bits(counts, n, L, B_max)
    m = min(bits)
    return max(i + 1 for i, v in enumerate(bits) if v == m)


def _sizes_index_term_in_bytes_per_bit(counts, n, L, B_max=16):
    desc = np.sort(np.asarray(counts, dtype=np.int64))[::-1]
    prefix = np.concatenate([[0], np.cumsum(desc, dtype=np.int64)])
    return [8 * (1 << B) * L + 8 * n * B + 8 * L * (n - int(prefix[min((1 << B) - 1, desc.size)]))
            for B in range(1, B_max + 1)]


MUTATIONS = {
    "ratio divides by cur": ("change_ratio", _ratio_over_cur),
    "ratio sign flipped": ("change_ratio", _ratio_wrong_sign),
    "bin rounds instead of floor": ("bin_ids", _bins_round),
    "anchor added instead of subtracted": ("bin_ids", _bins_anchor_sign),
    "zero minimum anchor kept as -0": ("grid_anchor", _anchor_keeps_signed_zero),
    "ties go to the larger bin": ("top_k", _topk_ties_to_larger),
    "indices in count order": ("top_k", _topk_count_order),
    "centre without the half bin": ("centres_of", _centres_no_half),
    "no value-space error check": ("assign_indices", _assign_no_check),
    "tolerance relative to prev": ("assign_indices", _assign_prev_tol),
    "bit packing MSB first": ("pack_block", _pack_msb_first),
    "elements per block off by one": ("elements_per_block", _epb_plus_one),
    "bin width E instead of 2E": ("grid_constants", _grid_width_E),
    "histogram counts non-binnable points": ("histogram", _hist_counts_all),
    "auto-B top 2^B bins": ("file_size_bits", _sizes_k_is_2_pow_B),
    "auto-B ties to the larger B": ("choose_B", _choose_B_ties_to_larger),
    "auto-B index table in bytes per bit": ("file_size_bits", _sizes_index_term_in_bytes_per_bit),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, monkeypatch):
    attr, fn = MUTATIONS[name]
    monkeypatch.setattr(O, attr, fn)
    assert _some_pin_fails(), f"no pin catches: {name}"
