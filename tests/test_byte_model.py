"""The key-switching byte model against the paper's Table "ks-param"
(Section V-B), stored as text in tests/golden/ks_param_table.txt."""
import os

import pytest

from paper_2512_18345_gb300 import roofline

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "ks_param_table.txt")
N = 1 << 16
MB = 1e6


def rows():
    out = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        v = line.split()
        out.append((int(v[0]), int(v[1]), int(v[2]), [float(x) for x in v[3:]]))
    return out


def close(model_mb, paper_mb):
    # the paper prints three significant figures
    return abs(model_mb - paper_mb) <= 0.006 * paper_mb + 0.05


@pytest.mark.parametrize("L,alpha,beta,vals", rows())
def test_footprints_match_paper(L, alpha, beta, vals):
    K = alpha
    assert roofline.beta_of(L, alpha) == beta
    f1, f3 = roofline.footprint_limbs(L, K, beta)
    W = roofline.limb_bytes(N)
    assert close(f1 * W / MB, vals[0]) and close(f3 * W / MB, vals[1])


@pytest.mark.parametrize("L,alpha,beta,vals", rows())
def test_traffic_against_paper(L, alpha, beta, vals):
    K = alpha
    W = roofline.limb_bytes(N)
    s1, s2, s3 = (x * W / MB for x in roofline.stage_limbs(L, K, beta))
    assert close(s2, vals[3])                                  # stage 2: every row
    # stage 1: the paper exceeds the model by exactly (beta - 1) L limbs
    assert close(s1 + (beta - 1) * L * W / MB, vals[2])
    if L <= 24:
        assert close(s3, vals[4])                              # stage 3: (24,12,2), (12,12,1)
    else:
        assert 0 < vals[4] - s3 < 75 * W / MB                  # (48,12,4): ~71 limbs unexplained


def test_limb_size_and_workload_figures():
    W = roofline.limb_bytes(N)
    assert W == 256 * 1024                                      # 0.25 MB per limb (Section II-A)
    assert 2 * 12 * W / 2 ** 20 == 6.0                          # 2 alpha limbs = 6 MB at alpha = 12 (Section IV-A)
    assert 4 * 60 * W / 2 ** 20 == 60.0                         # beta = 4 polys x 60 limbs = 60 MB (Section IV-A)
    # the build's main shape: l = 24, K = alpha = 8, beta = 3
    assert roofline.ks_bytes(N, 24, 8, 8) == 1224 * W
    assert roofline.ks_compulsory_hbm_bytes(N, 24, 8, 8) == 264 * W
