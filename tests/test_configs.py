"""Host-side workload configuration: packaging groups (Sec. 4.1)."""
import pytest

nt = pytest.importorskip("paper_2407_09543_gb300")


def test_packaging_groups():
    assert nt.configs.packaging_groups([1, 1, 4, 4]) == [[0, 1, 2, 3]]
    assert nt.configs.packaging_groups([1, 4, 1, 4, 4], "conservative") == [[0, 2], [1, 3, 4]]
    assert nt.configs.packaging_groups([4, 4], "conservative") == [[0, 1]]
    with pytest.raises(ValueError):
        nt.configs.packaging_groups([1], "other")
