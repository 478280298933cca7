"""Container for one evaluation problem: sources, centers, targets, pair lists."""
from dataclasses import dataclass, field
from typing import Optional

import numpy as np


@dataclass
class Geometry:
    """Arrays follow the library's layout.

    src_xyz (3, n_src) f64, src_weight (n_src,) f64, src_normal (3, n_src) f64,
    ctr_xyz (3, n_ctr) f64, ctr_radius (n_ctr,) f64, tgt_xyz (3, n_tgt) f64,
    tgt_center (n_tgt,) i32, tgt_normal (3, n_tgt) f64 or None,
    ctr_group (n_ctr,) i32, group_range_start (n_group+1,) i64,
    range_begin / range_end (nnz,) i32 -- half-open source index ranges.
    """
    src_xyz: np.ndarray
    src_weight: np.ndarray
    src_normal: Optional[np.ndarray]
    ctr_xyz: np.ndarray
    ctr_radius: np.ndarray
    tgt_xyz: np.ndarray
    tgt_center: np.ndarray
    tgt_normal: Optional[np.ndarray]
    ctr_group: np.ndarray
    group_range_start: np.ndarray
    range_begin: np.ndarray
    range_end: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def n_src(self):
        return int(self.src_weight.shape[0])

    @property
    def n_ctr(self):
        return int(self.ctr_xyz.shape[1])

    @property
    def n_tgt(self):
        return int(self.tgt_xyz.shape[1])

    @property
    def n_group(self):
        return int(self.group_range_start.shape[0] - 1)

    def group_source_counts(self):
        """Sources listed per group (duplicates counted)."""
        lens = (self.range_end.astype(np.int64) - self.range_begin.astype(np.int64))
        cs = np.concatenate([[0], np.cumsum(lens)])
        return cs[self.group_range_start[1:]] - cs[self.group_range_start[:-1]]

    def n_pairs(self):
        """Number of (target, source) pairs the lists define."""
        per_group = self.group_source_counts()
        return int(per_group[self.ctr_group[self.tgt_center]].sum())

    def subset_targets(self, idx):
        """A geometry restricted to the targets idx (sources, centers, lists kept)."""
        idx = np.asarray(idx, dtype=np.int64)
        return Geometry(self.src_xyz, self.src_weight, self.src_normal, self.ctr_xyz,
                        self.ctr_radius, np.ascontiguousarray(self.tgt_xyz[:, idx]),
                        np.ascontiguousarray(self.tgt_center[idx]),
                        None if self.tgt_normal is None else
                        np.ascontiguousarray(self.tgt_normal[:, idx]),
                        self.ctr_group, self.group_range_start, self.range_begin,
                        self.range_end, dict(self.meta))
