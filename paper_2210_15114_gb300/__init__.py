"""Implicit distance-matrix products on GB300 (sm_103a)."""
