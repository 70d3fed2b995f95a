"""Host bookkeeping of persisted Solve Factor tunings (no GPU): shape keys,
JSON round trip, rejection of malformed records, and installation through
the C ABI's tuning setter."""
import json

import pytest


@pytest.fixture(scope="module")
def mods():
    torch = pytest.importorskip("torch")
    from paper_1910_02371_gb300 import build as b
    b.build()
    from paper_1910_02371_gb300 import tc, tuning
    return torch, tc, tuning


def test_shape_keys_group_by_tier_and_powers_of_two(mods):
    torch, tc, tuning = mods
    k1 = tuning.shape_key(torch.float32, 16, 10_000, 10_000_000)
    k2 = tuning.shape_key(torch.float32, 13, 11_000, 10_500_000)   # same tier, same classes
    k3 = tuning.shape_key(torch.float32, 17, 10_000, 10_000_000)   # next tier
    assert k1 == k2 and k1 != k3
    assert tuning.shape_key(torch.float64, 16, 10_000, 10_000_000) != k1


def test_json_round_trip_and_apply(mods, tmp_path):
    torch, tc, tuning = mods
    key = tuning.shape_key(torch.float32, 32, 50_000, 50_000_000)
    tuning._records[key] = {"chunk_nnz": 1024, "batch_bytes": 0, "chol_rows_per_warp": 8, "ms": 1.5}
    path = str(tmp_path / "tune.json")
    tuning.save(path)
    tuning._records.clear()
    data = tuning.load(path)
    assert data[key]["chunk_nnz"] == 1024
    try:
        assert tuning.apply(torch.float32, 32, 50_000, 50_000_000)
        assert tc.get_solve_tuning(torch.float32, 32) == (1024, 0, 8, 0)
        assert not tuning.apply(torch.float32, 64, 50_000, 50_000_000)
    finally:
        tc.set_solve_tuning(torch.float32, 0, reset=True)
    bad = tmp_path / "bad.json"
    bad.write_text(json.dumps({"x": {"chunk_nnz": 1}}))
    with pytest.raises(ValueError):
        tuning.load(str(bad))


def test_setter_rejects_bad_values(mods):
    torch, tc, tuning = mods
    with pytest.raises(tc.TcError):
        tc.set_solve_tuning(torch.float32, 16, chol_rows_per_warp=3)
    with pytest.raises(tc.TcError):
        tc.set_solve_tuning(torch.float32, 16, chunk_nnz=-1)
    with pytest.raises(tc.TcError):
        tc.set_solve_tuning(torch.float32, 65)
    with pytest.raises(tc.TcError):
        tc.set_solve_tuning(torch.float32, 64, gram_kernel=3)


def test_record_without_gram_kernel_installs_the_automatic_engine(mods, tmp_path):
    """Records written before the Gram engine was a tuning dimension carry no
    gram_kernel: applying one installs the automatic engine (0); a record
    with one installs it."""
    torch, tc, tuning = mods
    k64 = tuning.shape_key(torch.float32, 64, 480_000, 100_000_000, "tf32_refine")
    k16 = tuning.shape_key(torch.float32, 16, 10_000, 10_000_000)
    path = tmp_path / "old.json"
    path.write_text(json.dumps({k16: {"chunk_nnz": 4096, "batch_bytes": 0, "chol_rows_per_warp": 8,
                                      "ms": 0.3},
                                k64: {"chunk_nnz": 0, "batch_bytes": 0, "chol_rows_per_warp": 0,
                                      "gram_kernel": tc.GRAM_WARP_MMA, "ms": 140.0}}))
    tuning._records.clear()
    tuning.load(str(path))
    try:
        assert tuning.apply(torch.float32, 16, 10_000, 10_000_000)
        assert tc.get_solve_tuning(torch.float32, 16) == (4096, 0, 8, 0)
        assert tuning.apply(torch.float32, 64, 480_000, 100_000_000, "tf32_refine")
        assert tc.get_solve_tuning(torch.float32, 64) == (0, 0, 0, tc.GRAM_WARP_MMA)
    finally:
        tc.set_solve_tuning(torch.float32, 0, reset=True)
        tuning._records.clear()
