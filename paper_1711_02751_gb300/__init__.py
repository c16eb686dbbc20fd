"""GB300 (sm_103a) implementation of the IMEX HDG-DG per-stage hot path for planar shallow water."""
