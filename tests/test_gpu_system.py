"""GPU build of A vs the oracle: index sets bit-exact, lengths bit-exact after
rounding the oracle's FP64 lengths to FP32, CSC = stable transpose."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import cuda, geometries

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,geom", geometries(), ids=[g[0] for g in geometries()])
def test_csr_and_csc_match_oracle(name, geom):
    cuda()
    from paper_1105_4002_gb300 import System
    A = oracle.system_matrix(geom)
    s = System(geom)
    assert (s.m, s.N, s.nnz) == (geom.m, geom.N, A.nnz)
    rp, col, val = s.export_csr()
    assert np.array_equal(rp, A.indptr.astype(np.int64))
    assert np.array_equal(col, A.indices)                  # same voxels, same traversal order
    assert np.array_equal(val, A.data.astype(np.float32))  # FP64 lengths rounded once
    C = A.tocsc()                                          # stable: rows ascending per column
    cp, row, cval = s.export_csc()
    assert np.array_equal(cp, C.indptr.astype(np.int64))
    assert np.array_equal(row, C.indices)
    assert np.array_equal(cval, C.data.astype(np.float32))
    s.close()


def test_full_size_64cubed_index_sets():
    cuda()
    from paper_1105_4002_gb300 import System
    geom = synth.get_config("c64").geometry()
    A = oracle.system_matrix(geom)
    s = System(geom)
    rp, col, val = s.export_csr()
    assert s.nnz == A.nnz
    assert np.array_equal(rp, A.indptr.astype(np.int64))
    assert np.array_equal(col, A.indices)
    assert np.array_equal(val, A.data.astype(np.float32))
    cp, row, cval = s.export_csc()
    C = A.tocsc()
    assert np.array_equal(cp, C.indptr.astype(np.int64))
    assert np.array_equal(row, C.indices)
    assert np.array_equal(cval, C.data.astype(np.float32))
    s.close()


def test_build_is_deterministic():
    cuda()
    from paper_1105_4002_gb300 import System
    geom = synth.get_config("c32").geometry()
    a = System(geom).export_csc()
    b = System(geom).export_csc()
    for u, v in zip(a, b):
        assert np.array_equal(u, v)


def test_invalid_geometry_is_rejected():
    cuda()
    from paper_1105_4002_gb300 import System, TVRError
    g = synth.cone_geometry(4, 2, 3, 12.0, 8.0)
    g.views[0, 0] = np.nan
    with pytest.raises(TVRError):
        System(g)


@pytest.mark.parametrize("storage", ["bf16", "u16"])
@pytest.mark.parametrize("name,geom", geometries(), ids=[g[0] for g in geometries()])
def test_16bit_codes_on_degenerate_scans(name, geom, storage):
    """The 16-bit storages on the same scans (one voxel, one ray, rays that miss
    the volume so rows are empty, odd sizes, axis-parallel rays): the same index
    sets, and values equal to the numpy emulation of their quantisation of the
    oracle's lengths, CSR and CSC alike."""
    cuda()
    from paper_1105_4002_gb300 import System
    from test_gpu_bf16 import effective as bf16_effective
    from test_gpu_u16 import effective as u16_effective
    A = oracle.system_matrix(geom)
    Ah, eff = (bf16_effective if storage == "bf16" else u16_effective)(A)
    s = System(geom, storage=storage)
    assert (s.m, s.N, s.nnz) == (geom.m, geom.N, A.nnz)
    rp, col, val = s.export_csr()
    assert np.array_equal(rp, A.indptr.astype(np.int64))
    assert np.array_equal(col, A.indices)
    assert np.array_equal(val, eff)
    C = Ah.tocsc()
    cp, row, cval = s.export_csc()
    assert np.array_equal(cp, C.indptr.astype(np.int64))
    assert np.array_equal(row, C.indices)
    assert np.array_equal(cval, C.data.astype(np.float32))
    s.close()
