"""FLARE mapped-SGP energy/force/uncertainty hot path for GB300 (sm_103a)."""
