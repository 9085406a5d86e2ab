"""Closed-loop discrete-time reachability with shared-slope CROWN Taylor models on B300 (sm_103a)."""
